"""Comparison of two Hamiltonians given as (x, z, c) (test infrastructure).

Tolerance: |c_gpu - c_oracle| <= REL * |c_oracle| + ABS (FP64 rounding of the
pair rotations).  Key sets must be equal, except for keys present on one side
only whose coefficient is

* within ABS of zero (a cancellation that one side rounds to an exact zero),
* within REL relative of the compression threshold eps, or
* within REL relative of one of ``thresholds``: the |C| of the term limit's
  cut (the max_terms-th largest |C|), where a key that ties with the threshold
  up to rounding may be kept on one side and dropped on the other.

No other difference is tolerated.
"""
import numpy as np

REL = 1e-12
ABS = 1e-14


def _keys(x, z):
    k = np.ascontiguousarray(np.concatenate([np.asarray(x, np.uint64).reshape(len(x), -1),
                                             np.asarray(z, np.uint64).reshape(len(z), -1)], 1))
    return k.view(np.dtype((np.void, k.shape[1] * 8))).ravel()


def as_dict(x, z, c):
    keys = np.concatenate([np.asarray(x, np.uint64), np.asarray(z, np.uint64)], 1)
    return {k.tobytes(): float(v) for k, v in zip(keys, np.asarray(c))}


def _excused(v, eps, thresholds, rel, abs_):
    a = np.abs(v)
    ok = a <= abs_
    if eps > 0:
        ok |= np.abs(a - eps) <= rel * eps + abs_
    for t in thresholds:
        ok |= np.abs(a - t) <= rel * t + abs_
    return ok


def compare(gpu, ref, eps=0.0, rel=REL, abs_=ABS, scale=None, thresholds=()):
    """Returns a list of mismatch descriptions (empty when equal)."""
    gx, gz, gc = gpu
    rx, rz, rc = ref
    gc = np.asarray(gc, np.float64)
    rc = np.asarray(rc, np.float64)
    if scale is not None:
        abs_ = abs_ * max(1.0, scale)
    gk, rk = _keys(gx, gz), _keys(rx, rz)
    bad = []
    for kind, keys in (("repeated_gpu_key", gk), ("repeated_oracle_key", rk)):
        u, cnt = np.unique(keys, return_counts=True)
        bad += [(kind, k.tobytes(), int(m)) for k, m in zip(u[cnt > 1], cnt[cnt > 1])]
    if bad:
        return bad
    if len(gk) == len(rk) and np.array_equal(gk, rk):
        ig = ir = np.arange(len(gk))
    else:
        _, ig, ir = np.intersect1d(gk, rk, assume_unique=True, return_indices=True)
        only_g = np.setdiff1d(np.arange(len(gk)), ig)
        only_r = np.setdiff1d(np.arange(len(rk)), ir)
        for kind, idx, keys, cs in (("only_gpu", only_g, gk, gc), ("only_oracle", only_r, rk, rc)):
            if len(idx):
                ok = _excused(cs[idx], eps, thresholds, rel, abs_)
                bad += [(kind, keys[i].tobytes(), float(cs[i])) for i in idx[~ok]]
    d = np.abs(gc[ig] - rc[ir])
    wrong = d > rel * np.abs(rc[ir]) + abs_
    bad += [("coef", gk[i].tobytes(), float(gc[i]), float(rc[j])) for i, j in zip(ig[wrong], ir[wrong])]
    return bad


def same_keys_exact(gpu, ref):
    gk, rk = _keys(*gpu[:2]), _keys(*ref[:2])
    return len(gk) == len(rk) and np.array_equal(np.sort(gk), np.sort(rk))


def cut_threshold(c, max_terms):
    """|C| of the max_terms-th largest coefficient: the term limit's threshold."""
    a = np.sort(np.abs(np.asarray(c, np.float64)))[::-1]
    return float(a[max_terms - 1]) if 0 < max_terms <= len(a) else 0.0
