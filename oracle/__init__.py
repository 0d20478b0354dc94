"""TEST INFRASTRUCTURE: ctypes wrapper of the plain CPU oracle (iqcc_oracle.cpp).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA
library (``paper_2603_08883_gb300``) and imports nothing from it.

All arrays follow the input layout: keys ``x``/``z`` as ``uint64[M, W]``
(qubit j = bit j%64 of word j//64), coefficients ``float64[M]``.  Sign
conventions are the library's: ``dress(P, tau)`` applies
e^{-i tau P/2} H e^{i tau P/2} and gradients are dE/dtau at tau = 0.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "iqcc_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (plain C++17, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        lib.orc_new.restype = vp
        lib.orc_new.argtypes = [ctypes.c_int]
        lib.orc_free.argtypes = [vp]
        lib.orc_size.restype = ctypes.c_int64
        lib.orc_size.argtypes = [vp]
        lib.orc_load.restype = ctypes.c_int
        lib.orc_load.argtypes = [vp, ctypes.c_int64, _u64p, _u64p, _f64p]
        lib.orc_export.restype = ctypes.c_int64
        lib.orc_export.argtypes = [vp, ctypes.c_int64, _u64p, _u64p, _f64p]
        lib.orc_dress.restype = ctypes.c_int
        lib.orc_dress.argtypes = [vp, _u64p, _u64p, ctypes.c_double]
        lib.orc_energy.restype = ctypes.c_double
        lib.orc_energy.argtypes = [vp, _f64p, _f64p]
        lib.orc_abc.argtypes = [vp, _u64p, _u64p, _f64p, _f64p, _f64p]
        lib.orc_gradient.restype = ctypes.c_double
        lib.orc_gradient.argtypes = [vp, _u64p, _u64p, _f64p, _f64p]
        lib.orc_dis.restype = ctypes.c_int64
        lib.orc_dis.argtypes = [vp, _f64p, _f64p, ctypes.c_int64, _u64p, _u64p, _f64p]
        lib.orc_prune.restype = ctypes.c_int64
        lib.orc_prune.argtypes = [vp, ctypes.c_double, ctypes.c_int64]
        lib.orc_energy_gradients.argtypes = [vp, vp, vp, ctypes.c_double, _f64p, _f64p, _f64p, _f64p, _f64p]
        lib.orc_energy_gradients.restype = ctypes.c_double
        lib.orc_iterate.restype = ctypes.c_int
        lib.orc_iterate.argtypes = [vp, _f64p, _f64p, ctypes.c_int, ctypes.c_int, _u64p, _u64p, _f64p,
                                    ctypes.c_double, ctypes.c_int64, _u64p, _u64p, _f64p, _f64p, _f64p,
                                    _i64p, _f64p]
        _lib = lib
    return _lib


def _u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(_u64p)


def _f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_f64p)


class Oracle:
    """A Hamiltonian held by the CPU oracle."""

    def __init__(self, n: int, x=None, z=None, c=None):
        self.n = int(n)
        self.W = (self.n + 63) // 64
        self._lib = _load()
        self._h = self._lib.orc_new(self.n)
        if not self._h:
            raise ValueError("bad qubit count")
        if x is not None:
            self.load(x, z, c)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.orc_free(h)
            self._h = None

    def _gen(self, gx, gz):
        gx = np.asarray(gx, dtype=np.uint64).reshape(self.W)
        gz = np.asarray(gz, dtype=np.uint64).reshape(self.W)
        return _u64(gx), _u64(gz)

    def _angles(self, theta, phi):
        t = np.asarray(theta, dtype=np.float64).reshape(self.n)
        p = np.asarray(phi, dtype=np.float64).reshape(self.n)
        return _f64(t), _f64(p)

    def load(self, x, z, c):
        x = np.asarray(x, dtype=np.uint64).reshape(-1, self.W)
        z = np.asarray(z, dtype=np.uint64).reshape(-1, self.W)
        (xa, xp), (za, zp), (ca, cp) = _u64(x), _u64(z), _f64(c)
        if not (len(xa) == len(za) == len(ca)):
            raise ValueError("length mismatch")
        self._lib.orc_load(self._h, len(ca), xp, zp, cp)

    def __len__(self):
        return int(self._lib.orc_size(self._h))

    def export(self):
        """(x, z, c) in canonical order (x big integer, then z)."""
        m = len(self)
        x = np.zeros((max(m, 1), self.W), np.uint64)
        z = np.zeros((max(m, 1), self.W), np.uint64)
        c = np.zeros(max(m, 1))
        self._lib.orc_export(self._h, m, x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                             c.ctypes.data_as(_f64p))
        return x[:m], z[:m], c[:m]

    def as_dict(self):
        x, z, c = self.export()
        return {tuple(np.concatenate([x[i], z[i]]).tolist()): float(c[i]) for i in range(len(c))}

    def dress(self, gx, gz, tau: float):
        (gxa, gxp), (gza, gzp) = self._gen(gx, gz)
        if self._lib.orc_dress(self._h, gxp, gzp, float(tau)) != 0:
            raise RuntimeError("oracle dress produced an imaginary coefficient")

    def energy(self, theta, phi) -> float:
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        return float(self._lib.orc_energy(self._h, tp, pp))

    def abc(self, gx, gz, theta, phi):
        (gxa, gxp), (gza, gzp) = self._gen(gx, gz)
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        out = np.zeros(3)
        self._lib.orc_abc(self._h, gxp, gzp, tp, pp, out.ctypes.data_as(_f64p))
        return out

    def gradient(self, gx, gz, theta, phi) -> float:
        (gxa, gxp), (gza, gzp) = self._gen(gx, gz)
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        return float(self._lib.orc_gradient(self._h, gxp, gzp, tp, pp))

    def energy_gradients(self, theta, phi, gx=None, gz=None, tau: float = 0.0):
        """E(tau) after the generator (gx, gz) at amplitude tau (none: E of H),
        dE/dtheta, dE/dphi (n each) and dE/dtau."""
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        dt = np.zeros(self.n)
        dp = np.zeros(self.n)
        dtau = np.zeros(1)
        if gx is None:
            gxp = gzp = None
        else:
            (gxa, gxp), (gza, gzp) = self._gen(gx, gz)
        e = self._lib.orc_energy_gradients(self._h, gxp, gzp, float(tau), tp, pp, dt.ctypes.data_as(_f64p),
                                           dp.ctypes.data_as(_f64p), dtau.ctypes.data_as(_f64p))
        if np.isnan(e):
            raise RuntimeError("oracle dress produced an imaginary coefficient")
        return float(e), dt, dp, float(dtau[0])

    def dis(self, theta, phi):
        """All DIS candidates, ordered: (cx, cz, g)."""
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        m = int(self._lib.orc_dis(self._h, tp, pp, 0, None, None, None))
        cx = np.zeros((max(m, 1), self.W), np.uint64)
        cz = np.zeros((max(m, 1), self.W), np.uint64)
        g = np.zeros(max(m, 1))
        self._lib.orc_dis(self._h, tp, pp, m, cx.ctypes.data_as(_u64p), cz.ctypes.data_as(_u64p),
                          g.ctypes.data_as(_f64p))
        return cx[:m], cz[:m], g[:m]

    def prune(self, eps: float, max_terms: int = 0) -> int:
        return int(self._lib.orc_prune(self._h, float(eps), int(max_terms)))

    def iterate(self, theta, phi, n_gen: int, eps: float = 0.0, max_terms: int = 0,
                forced_x=None, forced_z=None, forced_tau=None):
        """One iQCC iteration; returns a dict with the generators, g, tau, abc, E."""
        (ta, tp), (pa, pp) = self._angles(theta, phi)
        W = self.W
        nf = 0
        fx = fz = None
        fxp = fzp = None
        if forced_x is not None:
            fx, fxp = _u64(np.asarray(forced_x, np.uint64).reshape(-1, W))
            fz, fzp = _u64(np.asarray(forced_z, np.uint64).reshape(-1, W))
            nf = len(fx)
            n_gen = nf
        ftp = None
        if forced_tau is not None:
            fta, ftp = _f64(np.asarray(forced_tau, np.float64).reshape(n_gen))
        gx = np.zeros((max(n_gen, 1), W), np.uint64)
        gz = np.zeros((max(n_gen, 1), W), np.uint64)
        g = np.zeros(max(n_gen, 1))
        tau = np.zeros(max(n_gen, 1))
        abc = np.zeros((max(n_gen, 1), 3))
        removed = ctypes.c_int64(0)
        energy = ctypes.c_double(0.0)
        used = self._lib.orc_iterate(self._h, tp, pp, int(n_gen), nf, fxp, fzp, ftp, float(eps),
                                     int(max_terms), gx.ctypes.data_as(_u64p), gz.ctypes.data_as(_u64p),
                                     g.ctypes.data_as(_f64p), tau.ctypes.data_as(_f64p),
                                     abc.ctypes.data_as(_f64p), ctypes.byref(removed), ctypes.byref(energy))
        if used < 0:
            raise RuntimeError("oracle iteration failed")
        return {"gx": gx[:used], "gz": gz[:used], "g": g[:used], "tau": tau[:used], "abc": abc[:used],
                "removed": int(removed.value), "energy": float(energy.value), "M": len(self)}
