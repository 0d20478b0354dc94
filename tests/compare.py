"""Comparison of two Hamiltonians given as (x, z, c) (test infrastructure).

Tolerance: |c_gpu - c_oracle| <= REL * |c_oracle| + ABS (FP64 rounding of the
pair rotations; the same floor applies to the key-set comparison: keys whose
coefficient is within ABS of zero on both sides, or within REL of the
compression threshold, may differ).
"""
import numpy as np

REL = 1e-12
ABS = 1e-14


def as_dict(x, z, c):
    keys = np.concatenate([np.asarray(x, np.uint64), np.asarray(z, np.uint64)], 1)
    return {k.tobytes(): float(v) for k, v in zip(keys, np.asarray(c))}


def compare(gpu, ref, eps=0.0, rel=REL, abs_=ABS, scale=None):
    """Returns a list of mismatch descriptions (empty when equal)."""
    g = as_dict(*gpu)
    o = as_dict(*ref)
    bad = []
    if scale is not None:
        abs_ = abs_ * max(1.0, scale)
    for k in g.keys() | o.keys():
        cg, co = g.get(k), o.get(k)
        if cg is None or co is None:
            v = cg if co is None else co
            near_zero = abs(v) <= abs_
            near_thr = eps > 0 and abs(abs(v) - eps) <= rel * eps + abs_
            if not (near_zero or near_thr):
                bad.append(("only_gpu" if co is None else "only_oracle", k, v))
            continue
        if abs(cg - co) > rel * abs(co) + abs_:
            bad.append(("coef", k, cg, co))
    return bad


def same_keys_exact(gpu, ref):
    return set(as_dict(*gpu)) == set(as_dict(*ref))
