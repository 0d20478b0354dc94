"""Seeded synthetic inputs for the iQCC dressing path.

This module only *generates inputs*: molecular-integral-shaped random tensors,
their Jordan-Wigner qubit Hamiltonian (Eq. 1 -> Eq. 2, App. A Eq. 8 -> Eq. 9),
random real Pauli Hamiltonians for edge cases, and QMF reference angles
(Eq. 3 / Eq. 10).  Both the CUDA library and the CPU oracle consume what it
returns; it contains none of the dressing, energy or gradient arithmetic.

Key layout of every Hamiltonian returned here: ``x`` and ``z`` are
``uint64[M, W]`` with ``W = ceil(n/64)``; qubit ``j`` is bit ``j % 64`` of word
``j // 64``; letter (x,z) = (0,0) I, (1,0) X, (1,1) Y, (0,1) Z; ``c`` is
``float64[M]``.  The paper's Ru-catalyst integral files are not available, so
the recipes below stand in for them at the paper's qubit counts.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hamgen.c")
_LIB = os.path.join(_HERE, "libhamgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the Jordan-Wigner generator (plain C, host only)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.hamgen_jw.restype = ctypes.c_longlong
        lib.hamgen_jw.argtypes = [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                  ctypes.POINTER(ctypes.POINTER(ctypes.c_uint64))]
        lib.hamgen_free.argtypes = [ctypes.c_void_p]
        _lib = lib
    return _lib


def n_words(n: int) -> int:
    return (n + 63) // 64


# ---------------------------------------------------------------------------
# integrals
# ---------------------------------------------------------------------------

def _canonical_quadruples(norb: int) -> np.ndarray:
    """All (p,q,r,s) with p>=q, r>=s and pair(pq) >= pair(rs), lexicographic."""
    p, q = np.tril_indices(norb)
    pair = np.stack([p, q], 1)                   # pairs in lexicographic order
    a, b = np.tril_indices(len(pair))            # pair index a >= b
    return np.concatenate([pair[a], pair[b]], 1)


def _fill_eri(norb: int, quads: np.ndarray, vals: np.ndarray) -> np.ndarray:
    eri = np.zeros((norb,) * 4)
    p, q, r, s = quads.T
    for (i, j, k, l) in ((p, q, r, s), (q, p, r, s), (p, q, s, r), (q, p, s, r),
                         (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)):
        eri[i, j, k, l] = vals
    return eri


def _sym_one_body(rng, norb: int, scale: np.ndarray | float) -> np.ndarray:
    p, q = np.triu_indices(norb)
    v = rng.standard_normal(len(p))
    h = np.zeros((norb, norb))
    h[p, q] = v
    h[q, p] = v
    return h * scale


def integrals(kind: str, norb: int, seed: int):
    """Seeded real integrals ``h[p,q]`` and chemist ``eri[p,q,r,s] = (pq|rs)``.

    kind:
      * ``"plain"``  - h ~ N(0,1), (pq|rs) ~ N(0,0.1) (standard deviations).
      * ``"decay"``  - as plain, times exp(-|p-q|/3) for h and
        exp(-(|p-q|+|r-s|)/3) for (pq|rs), which keeps the 8-fold symmetry.
      * ``"dblock"`` - decay background with sigma 0.05 for (pq|rs), and a
        strongly coupled block of 10 orbitals starting at norb*2//5 where all
        four indices fall inside it, drawn from N(0, 0.5).
    The upper triangle of h is drawn first, then the canonical quadruples of
    (pq|rs) in lexicographic order, all from ``Generator(PCG64(seed))``.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.arange(norb)
    dist = np.abs(idx[:, None] - idx[None, :]).astype(float)
    if kind == "plain":
        h = _sym_one_body(rng, norb, 1.0)
        quads = _canonical_quadruples(norb)
        vals = 0.1 * rng.standard_normal(len(quads))
    elif kind in ("decay", "dblock"):
        h = _sym_one_body(rng, norb, np.exp(-dist / 3.0))
        quads = _canonical_quadruples(norb)
        p, q, r, s = quads.T
        decay = np.exp(-(np.abs(p - q) + np.abs(r - s)) / 3.0)
        sigma = 0.1 if kind == "decay" else 0.05
        vals = sigma * decay * rng.standard_normal(len(quads))
        if kind == "dblock":
            lo = (norb * 2) // 5
            hi = lo + min(10, norb - lo)
            inside = (p >= lo) & (p < hi) & (q >= lo) & (q < hi) & (r >= lo) & (r < hi) & (s >= lo) & (s < hi)
            vals = np.where(inside, 0.5 * rng.standard_normal(len(quads)), vals)
    else:
        raise ValueError(f"unknown integral kind {kind!r}")
    return h, _fill_eri(norb, quads, vals)


def jordan_wigner(h: np.ndarray, eri: np.ndarray, rel_drop: float = 1e-14):
    """Qubit Hamiltonian of the integrals: (n, x, z, c), unique keys in a fixed order.

    Strings with |c| < rel_drop * max|c| are dropped.
    """
    norb = h.shape[0]
    n = 2 * norb
    W = n_words(n)
    lib = _load()
    h = np.ascontiguousarray(h, dtype=np.float64)
    eri = np.ascontiguousarray(eri, dtype=np.float64)
    out = ctypes.POINTER(ctypes.c_uint64)()
    M = lib.hamgen_jw(norb, h.ctypes.data, eri.ctypes.data, rel_drop, ctypes.byref(out))
    if M < 0:
        raise RuntimeError("hamgen_jw failed")
    L = 2 * W + 1
    try:
        rows = np.ctypeslib.as_array(out, shape=(max(M, 1) * L,))[: M * L].reshape(M, L).copy()
    finally:
        lib.hamgen_free(out)
    x = np.ascontiguousarray(rows[:, :W])
    z = np.ascontiguousarray(rows[:, W:2 * W])
    c = rows[:, 2 * W].view(np.float64).copy()
    return n, x, z, c


# ---------------------------------------------------------------------------
# random real Pauli Hamiltonians (edge cases, ragged word counts)
# ---------------------------------------------------------------------------

def _mask_top(a: np.ndarray, n: int) -> np.ndarray:
    W = a.shape[1]
    r = n - 64 * (W - 1)
    if r < 64:
        a[:, W - 1] &= np.uint64((1 << r) - 1)
    return a


def random_pauli_strings(n: int, m: int, rng, density: float = 0.5, even_y: bool = True):
    """``m`` random Pauli keys on ``n`` qubits (uint64[m, W] x and z).

    Each qubit is non-identity with probability ``density``; with ``even_y``
    every string has an even number of Y letters (real, symmetric strings).
    """
    W = n_words(n)
    act = rng.random((m, n)) < density
    let = rng.integers(1, 4, size=(m, n))          # 1 X, 2 Y, 3 Z
    xb = act & ((let == 1) | (let == 2))
    zb = act & ((let == 2) | (let == 3))
    if even_y:
        ny = (xb & zb).sum(1)
        odd = np.nonzero(ny & 1)[0]
        for i in odd:                                 # turn the first Y into X
            j = np.nonzero(xb[i] & zb[i])[0][0]
            zb[i, j] = False
    return _pack(xb, W), _pack(zb, W)


def _pack(bits: np.ndarray, W: int) -> np.ndarray:
    m, n = bits.shape
    out = np.zeros((m, W), dtype=np.uint64)
    for j in range(n):
        out[:, j // 64] |= bits[:, j].astype(np.uint64) << np.uint64(j % 64)
    return out


def random_hamiltonian(n: int, m: int, seed: int, density: float = 0.5, scale: str = "lognormal",
                       unique: bool = True):
    """Random real Hamiltonian: (n, x, z, c).  Keys unique when ``unique``."""
    rng = np.random.Generator(np.random.PCG64(seed))
    x, z = random_pauli_strings(n, m, rng, density)
    if unique and m:
        key = np.concatenate([x, z], 1)
        _, first = np.unique(key, axis=0, return_index=True)
        first.sort()
        x, z = x[first], z[first]
    k = len(x)
    if scale == "lognormal":
        c = rng.standard_normal(k) * np.exp(rng.uniform(-12.0, 1.0, k))
    else:
        c = rng.standard_normal(k)
    return n, np.ascontiguousarray(x), np.ascontiguousarray(z), c


def random_generator(n: int, rng, weight: int | None = None):
    """A random Hermitian Pauli generator with an odd number of Y letters."""
    W = n_words(n)
    weight = weight or int(rng.integers(1, min(n, 6) + 1))
    sites = rng.choice(n, size=min(weight, n), replace=False)
    xb = np.zeros((1, n), bool)
    zb = np.zeros((1, n), bool)
    for j in sites:
        l = int(rng.integers(1, 4))
        xb[0, j] = l in (1, 2)
        zb[0, j] = l in (2, 3)
    if ((xb & zb).sum() & 1) == 0:                    # make #Y odd
        j = int(sites[0])
        if xb[0, j] and zb[0, j]:
            zb[0, j] = False                          # Y -> X
        else:
            xb[0, j] = True
            zb[0, j] = True                           # -> Y
    return _pack(xb, W)[0], _pack(zb, W)[0]


# ---------------------------------------------------------------------------
# QMF reference angles
# ---------------------------------------------------------------------------

def qmf_angles(n: int, kind: str, seed: int = 0):
    """QMF Bloch angles (theta, phi), float64[n] each.

    ``"uniform"``: theta ~ U[0, pi), phi ~ U[0, 2 pi) from PCG64([seed, 1]).
    ``"basis"``: theta = pi on qubits 0 .. n/2-1 (occupied), 0 elsewhere, phi = 0.
    """
    if kind == "uniform":
        rng = np.random.Generator(np.random.PCG64([seed, 1]))
        return rng.uniform(0.0, np.pi, n), rng.uniform(0.0, 2.0 * np.pi, n)
    if kind == "basis":
        theta = np.zeros(n)
        theta[: n // 2] = np.pi
        return theta, np.zeros(n)
    raise ValueError(kind)


# ---------------------------------------------------------------------------
# workloads at the paper's sizes
# ---------------------------------------------------------------------------

@dataclass(frozen=True)
class Workload:
    name: str
    seed: int
    norb: int
    integrals: str
    angles: str
    n_iter: int
    n_gen: int
    eps: float
    max_terms: int                 # term limit after every dress; <= 0: none
    capacity: int                  # admission limit in rows (2 x max_terms covers one dress)
    notes: str = field(default="")

    @property
    def n_qubits(self) -> int:
        return 2 * self.norb


WORKLOADS = {
    "jw8": Workload("jw8", 8, 4, "plain", "uniform", 3, 2, 0.0, 0, 1 << 14,
                    "8 qubits, 4 orbitals, random QMF angles, no pruning"),
    "jw24": Workload("jw24", 24, 12, "decay", "basis", 20, 4, 1e-10, 0, 1 << 30,
                     "24 qubits, 12 orbitals with exp(-d/3) decay, prune 1e-10"),
    "jw100": Workload("jw100", 100, 50, "dblock", "basis", 10, 8, 1e-8, 800_000_000, 1_600_000_000,
                      "100 qubits, 50 orbitals, strongly coupled 10-orbital block, prune 1e-8, "
                      "term cap 8e8"),
}


def workload_hamiltonian(w: Workload):
    h, eri = integrals(w.integrals, w.norb, w.seed)
    return jordan_wigner(h, eri)


def workload_angles(w: Workload):
    return qmf_angles(w.n_qubits, w.angles, w.seed)
