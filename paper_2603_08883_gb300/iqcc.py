"""Python binding of libiqcc.so (ctypes; argument marshalling only).

Every function below has the name of the C entry point it calls (see
``include/iqcc.h``) and does no arithmetic of the method itself.  PyTorch, when
present, supplies the CUDA stream (and, on request, the device allocator) to
the library.  There is no CPU fallback: importing this module
raises when the compiled library is missing, and creating a Hamiltonian raises
when no CUDA device is visible.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libiqcc.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with `python -m paper_2603_08883_gb300.build` "
                      "(the iQCC path has no CPU fallback)")

_lib = ctypes.CDLL(LIB_PATH)

_u64p = ctypes.POINTER(ctypes.c_uint64)
_f64p = ctypes.POINTER(ctypes.c_double)
_f32p = ctypes.POINTER(ctypes.c_float)
_i64p = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

STATUS = {0: "IQCC_OK", 1: "IQCC_ERR_ARG", 2: "IQCC_ERR_CUDA", 3: "IQCC_ERR_OOM", 4: "IQCC_ERR_CAPACITY",
          5: "IQCC_ERR_HASH_FULL", 6: "IQCC_ERR_TIMEOUT", 7: "IQCC_ERR_STATE"}


class IqccError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status


class iqcc_opts(ctypes.Structure):
    _fields_ = [("n_qubits", ctypes.c_int), ("capacity", ctypes.c_int64), ("max_probe", ctypes.c_int),
                ("stream", ctypes.c_void_p), ("alloc", ALLOC_FN), ("free", FREE_FN), ("alloc_user", ctypes.c_void_p)]


class iqcc_iter_opts(ctypes.Structure):
    _fields_ = [("n_gen", ctypes.c_int), ("eps", ctypes.c_double), ("max_terms", ctypes.c_int64),
                ("min_gradient", ctypes.c_double), ("n_forced", ctypes.c_int), ("forced_x", _u64p),
                ("forced_z", _u64p), ("forced_tau", _f64p), ("screening", ctypes.c_int)]


class iqcc_iter_result(ctypes.Structure):
    _fields_ = [("n_applied", ctypes.c_int), ("gx", ctypes.c_uint64 * 256), ("gz", ctypes.c_uint64 * 256),
                ("grad", ctypes.c_double * 64), ("tau", ctypes.c_double * 64), ("abc", (ctypes.c_double * 3) * 64),
                ("n_terms_before", ctypes.c_int64), ("n_terms_peak", ctypes.c_int64), ("n_removed", ctypes.c_int64),
                ("n_terms", ctypes.c_int64), ("dressed_terms", ctypes.c_int64), ("energy", ctypes.c_double)]


class iqcc_stats(ctypes.Structure):
    _fields_ = [("n_dress", ctypes.c_int64), ("dressed_terms", ctypes.c_int64), ("anticommuting", ctypes.c_int64),
                ("appended", ctypes.c_int64), ("dress_kernel_ms", ctypes.c_double), ("dress_bytes", ctypes.c_double),
                ("n_energy", ctypes.c_int64), ("energy_kernel_ms", ctypes.c_double),
                ("energy_bytes", ctypes.c_double), ("prune_ms", ctypes.c_double), ("dis_ms", ctypes.c_double),
                ("hash_ms", ctypes.c_double), ("hash_rebuilds", ctypes.c_int64), ("rows_allocated", ctypes.c_int64),
                ("hash_slots", ctypes.c_int64), ("kernel_launches", ctypes.c_int64),
                ("n_sorted_groups", ctypes.c_int64), ("sorted_dress_ms", ctypes.c_double),
                ("screen_terms", ctypes.c_int64), ("screen_ms", ctypes.c_double), ("words", ctypes.c_int),
                ("pad", ctypes.c_int), ("fixed_bin_dresses", ctypes.c_int64), ("bin_overflows", ctypes.c_int64)]


def _sig(name, res, args):
    f = getattr(_lib, name)
    f.restype = res
    f.argtypes = args
    return f


_c = ctypes.c_int
_load = _sig("iqcc_load_hamiltonian", _c, [ctypes.POINTER(_vp), ctypes.POINTER(iqcc_opts), ctypes.c_int64, _u64p,
                                           _u64p, _f64p])
_dress = _sig("iqcc_dress", _c, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, ctypes.POINTER(ctypes.c_int)])
_cross_rows = _sig("iqcc_cross_rows", _c, [_vp, _u64p, _u64p, ctypes.c_int64, _i64p, _u64p, _u64p, _f64p])
_dress_cross = _sig("iqcc_dress_cross", _c, [_vp, _u64p, _u64p, ctypes.c_double, ctypes.c_int64, _u64p, _u64p,
                                             _f64p])
_set_model = _sig("iqcc_set_screening_model", _c, [_vp, _f32p, _f32p, _f32p, _f32p, _f32p, ctypes.c_float])
_set_floor = _sig("iqcc_set_screening_floor", _c, [_vp, ctypes.c_double])
_features = _sig("iqcc_term_features", _c, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, _f64p, _f32p])
_future = _sig("iqcc_future_energies", _c, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, _f64p, _f64p, _f64p])
_scores = _sig("iqcc_term_scores", _c, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, _f64p, _f32p])
_prune_learned = _sig("iqcc_prune_learned", _c, [_vp, ctypes.c_double, ctypes.c_int64, ctypes.c_int, _u64p, _u64p,
                                                 _f64p, _f64p, _i64p])
_dress_sorted = _sig("iqcc_dress_sorted", _c, [_vp, ctypes.c_int, _u64p, _u64p, _f64p, ctypes.c_int,
                                               ctypes.POINTER(ctypes.c_int)])
_prune = _sig("iqcc_prune", _c, [_vp, ctypes.c_double, ctypes.c_int64, _i64p])
_dress_pair_raw = _sig("iqcc_dress_pair", _c, [_vp, _vp, _u64p, _u64p, ctypes.c_double, _u64p, _u64p, _u64p, _u64p])


def _dress_pair(a, b, gx, gz, mx, mz, ax, az, tau):
    return _dress_pair_raw(a, b, gx, gz, tau, mx, mz, ax, az)


_abc_parts = _sig("iqcc_generator_abc_parts", _c, [ctypes.POINTER(_vp), ctypes.c_int, _u64p, _u64p, _f64p, _f64p,
                                                   _f64p, _f64p])
_prune_parts = _sig("iqcc_prune_parts", _c, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                                               _i64p])
_energy = _sig("iqcc_qmf_energy", _c, [_vp, _f64p, _f64p, _f64p])
_abc = _sig("iqcc_generator_abc", _c, [_vp, _u64p, _u64p, _f64p, _f64p, _f64p])
_egrad = _sig("iqcc_energy_gradients", _c, [_vp, _u64p, _u64p, ctypes.c_double, _f64p, _f64p, _f64p, _f64p, _f64p,
                                            _f64p])
_dis = _sig("iqcc_dis_gradients", _c, [_vp, _f64p, _f64p, ctypes.c_int64, _u64p, _u64p, ctypes.c_int64, _i64p,
                                       _u64p, _u64p, _f64p])
_iterate = _sig("iqcc_iterate", _c, [_vp, _f64p, _f64p, ctypes.POINTER(iqcc_iter_opts),
                                     ctypes.POINTER(iqcc_iter_result)])
_num = _sig("iqcc_num_terms", _c, [_vp, _i64p])
_export = _sig("iqcc_export", _c, [_vp, ctypes.c_int64, _i64p, _u64p, _u64p, _f64p])
_export_rows = _sig("iqcc_export_rows", _c, [_vp, ctypes.c_int64, _i64p, _u64p, _u64p, _f64p])
_bin_slack = _sig("iqcc_set_bin_slack", _c, [_vp, ctypes.c_double, ctypes.c_int])
_stats = _sig("iqcc_get_stats", _c, [_vp, ctypes.POINTER(iqcc_stats)])
_reset = _sig("iqcc_reset_stats", _c, [_vp])
_err = _sig("iqcc_last_error", ctypes.c_char_p, [_vp])
_free = _sig("iqcc_free", None, [_vp])
_set_wait = _sig("iqcc_set_wait_limit", _c, [_vp, ctypes.c_int])
_wait_selftest = _sig("iqcc_wait_selftest", _c, [_vp])
_energy_noalloc = _sig("iqcc_qmf_energy_noalloc", _c, [ctypes.c_int, ctypes.c_int64, _vp, _vp, _f64p, _f64p, _vp,
                                                       _f64p])


def _u64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    if shape is not None:
        a = a.reshape(shape)
    return a, a.ctypes.data_as(_u64p)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a, a.ctypes.data_as(_f64p)


def _torch_hooks(device, torch_alloc):
    """(stream handle, alloc callback, free callback) from PyTorch, or Nones.
    The stream is PyTorch's current stream; device memory comes from PyTorch's
    caching allocator only when ``torch_alloc`` (else the library's cudaMalloc,
    which returns freed memory to the device at once)."""
    try:
        import torch
    except ImportError:
        return None, None, None
    if not torch.cuda.is_available():
        return None, None, None
    dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream(dev)
    if not torch_alloc:
        return stream.cuda_stream, None, None

    def _alloc(size, _user):
        try:
            return torch.cuda.caching_allocator_alloc(int(size), dev.index, stream)
        except Exception:  # out of memory -> NULL, the library reports IQCC_ERR_OOM
            return None

    def _free(ptr, _user):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    return stream.cuda_stream, ALLOC_FN(_alloc), FREE_FN(_free)


class Hamiltonian:
    """A Hamiltonian resident on the GPU (an ``iqcc_ctx``)."""

    def __init__(self, handle, n, keepalive):
        self._h = handle
        self.n = n
        self.W = (n + 63) // 64
        self._keepalive = keepalive

    def _check(self, st):
        if st != 0:
            raise IqccError(st, _err(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _free(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __len__(self):
        return iqcc_num_terms(self)

    @property
    def handle(self):
        return self._h


def iqcc_load_hamiltonian(n_qubits: int, x, z, coef, capacity: int = 0, max_probe: int = 0,
                          use_torch: bool = True, device=None, torch_alloc: bool = False) -> Hamiltonian:
    """Load H = sum_k coef[k] P(x[k], z[k]) onto the GPU (iqcc_load_hamiltonian).
    With ``use_torch`` the library runs on PyTorch's current stream."""
    W = (n_qubits + 63) // 64
    xa, xp = _u64(x, (-1, W))
    za, zp = _u64(z, (-1, W))
    ca, cp = _f64(coef)
    if not (len(xa) == len(za) == len(ca)):
        raise ValueError("x, z and coef lengths differ")
    stream, alloc, free = _torch_hooks(device, torch_alloc) if use_torch else (None, None, None)
    opts = iqcc_opts(n_qubits, capacity, max_probe, stream, alloc or ALLOC_FN(), free or FREE_FN(), None)
    h = _vp()
    st = _load(ctypes.byref(h), ctypes.byref(opts), len(ca), xp, zp, cp)
    if st != 0:
        raise IqccError(st, _err(None).decode())
    return Hamiltonian(h, n_qubits, (alloc, free, opts))


def iqcc_dress(H: Hamiltonian, gx, gz, tau) -> int:
    gxa, gxp = _u64(gx, (-1, H.W))
    gza, gzp = _u64(gz, (-1, H.W))
    ta, tp = _f64(np.atleast_1d(tau), len(gxa))
    applied = ctypes.c_int(0)
    H._check(_dress(H._h, len(gxa), gxp, gzp, tp, ctypes.byref(applied)))
    return applied.value


def iqcc_cross_rows(H: Hamiltonian, gx, gz):
    """The rows that anticommute with P, for the peer partition: (x [k, W], z [k, W], c [k])."""
    gxa, gxp = _u64(gx, (H.W,))
    gza, gzp = _u64(gz, (H.W,))
    n = ctypes.c_int64(0)
    H._check(_cross_rows(H._h, gxp, gzp, 0, ctypes.byref(n), None, None, None))
    k = n.value
    x = np.zeros((max(k, 1), H.W), np.uint64)
    z = np.zeros((max(k, 1), H.W), np.uint64)
    c = np.zeros(max(k, 1))
    H._check(_cross_rows(H._h, gxp, gzp, k, ctypes.byref(n), x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                         c.ctypes.data_as(_f64p)))
    return x[:k], z[:k], c[:k]


def iqcc_dress_cross(H: Hamiltonian, gx, gz, tau: float, px, pz, pc) -> None:
    """Dress by P given the peer partition's anticommuting rows (from iqcc_cross_rows on the peer)."""
    gxa, gxp = _u64(gx, (H.W,))
    gza, gzp = _u64(gz, (H.W,))
    pxa, pxp = _u64(px, (-1, H.W))
    pza, pzp = _u64(pz, (-1, H.W))
    pca, pcp = _f64(pc, len(pxa))
    H._check(_dress_cross(H._h, gxp, gzp, float(tau), len(pxa), pxp, pzp, pcp))


def iqcc_dress_sorted(H: Hamiltonian, gx, gz, tau, fuse: int = 1) -> int:
    gxa, gxp = _u64(gx, (-1, H.W))
    gza, gzp = _u64(gz, (-1, H.W))
    ta, tp = _f64(np.atleast_1d(tau), len(gxa))
    applied = ctypes.c_int(0)
    H._check(_dress_sorted(H._h, len(gxa), gxp, gzp, tp, int(fuse), ctypes.byref(applied)))
    return applied.value


def _gens(H, gx, gz):
    if gx is None:
        return 0, None, None, []
    gxa, gxp = _u64(gx, (-1, H.W))
    gza, gzp = _u64(gz, (-1, H.W))
    return len(gxa), gxp, gzp, [gxa, gza]


def iqcc_set_screening_model(H: Hamiltonian, w1, b1, w2, b2, w3, b3: float) -> None:
    """Perceptron weights: w1 [256, 8], b1 [256], w2 [256, 256] (out, in), b2 [256], w3 [256], b3."""
    arrs = [np.ascontiguousarray(a, np.float32).reshape(-1) for a in (w1, b1, w2, b2, w3)]
    if [a.size for a in arrs] != [256 * 8, 256, 256 * 256, 256, 256]:
        raise ValueError("weight shapes: w1 [256, 8], b1 [256], w2 [256, 256], b2 [256], w3 [256]")
    H._check(_set_model(H._h, *[a.ctypes.data_as(_f32p) for a in arrs], float(b3)))


def iqcc_set_screening_floor(H: Hamiltonian, frac: float) -> None:
    """Share of the learned term limit kept by largest |C| first (0..1; 0.5 by default)."""
    H._check(_set_floor(H._h, float(frac)))


def iqcc_term_features(H: Hamiltonian, theta, phi, gx=None, gz=None) -> np.ndarray:
    """Screening features of every term (rows in iqcc_export order): float32 [M, 8]."""
    k, gxp, gzp, keep = _gens(H, gx, gz)
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    out = np.zeros((len(H), 8), np.float32)
    H._check(_features(H._h, k, gxp, gzp, tp, pp, out.ctypes.data_as(_f32p)))
    return out


def iqcc_future_energies(H: Hamiltonian, theta, phi, gx, gz, tau) -> np.ndarray:
    """E_fut of every term after the generators (<= 8) at amplitudes tau (iqcc_export order)."""
    k, gxp, gzp, keep = _gens(H, gx, gz)
    ta, tp = _f64(np.atleast_1d(tau), k)
    tha, thp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    out = np.zeros(len(H))
    H._check(_future(H._h, k, gxp, gzp, tp, thp, pp, out.ctypes.data_as(_f64p)))
    return out


def iqcc_term_scores(H: Hamiltonian, theta, phi, gx=None, gz=None) -> np.ndarray:
    """The screening model's score of every term (iqcc_export order): float32 [M]."""
    k, gxp, gzp, keep = _gens(H, gx, gz)
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    out = np.zeros(len(H), np.float32)
    H._check(_scores(H._h, k, gxp, gzp, tp, pp, out.ctypes.data_as(_f32p)))
    return out


def iqcc_prune_learned(H: Hamiltonian, eps: float, max_terms: int, theta, phi, gx=None, gz=None) -> int:
    k, gxp, gzp, keep = _gens(H, gx, gz)
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    removed = ctypes.c_int64(0)
    H._check(_prune_learned(H._h, float(eps), int(max_terms), k, gxp, gzp, tp, pp, ctypes.byref(removed)))
    return removed.value


def iqcc_prune(H: Hamiltonian, eps: float, max_terms: int = 0) -> int:
    removed = ctypes.c_int64(0)
    H._check(_prune(H._h, float(eps), int(max_terms), ctypes.byref(removed)))
    return removed.value


def iqcc_dress_pair(A: Hamiltonian, B: Hamiltonian, gx, gz, tau: float, mx, mz, ax, az) -> None:
    """iqcc_dress_pair: dress two partitions of one Hamiltonian (A's keys have
    (ax, az) under the masks (mx, mz)) by one generator on the device."""
    W = A.W
    arrs = [_u64(v, (W,)) for v in (gx, gz, mx, mz, ax, az)]
    st = _dress_pair(A._h, B._h, *[p for _, p in arrs], float(tau))
    if st != 0:
        msg = _err(A._h).decode()
        raise IqccError(st, msg if msg != "no error" else _err(B._h).decode())


def iqcc_generator_abc_parts(parts, gx, gz, theta, phi):
    """iqcc_generator_abc_parts: (A, B, C) summed over the parts and the
    minimising amplitude tau* of the summed E(tau)."""
    parts = list(parts)
    W = parts[0].W
    gxa, gxp = _u64(gx, (W,))
    gza, gzp = _u64(gz, (W,))
    ta, tp = _f64(theta, parts[0].n)
    pa, pp = _f64(phi, parts[0].n)
    arr = (_vp * len(parts))(*[H._h for H in parts])
    abc = np.zeros(3)
    tau = ctypes.c_double(0.0)
    st = _abc_parts(arr, len(parts), gxp, gzp, tp, pp, abc.ctypes.data_as(_f64p), ctypes.byref(tau))
    if st != 0:
        msgs = [_err(H._h).decode() for H in parts if H._h]
        raise IqccError(st, next((m for m in msgs if m != "no error"), _err(None).decode()))
    return tuple(float(v) for v in abc), tau.value


def iqcc_prune_parts(parts, eps: float, max_terms: int = 0) -> int:
    """iqcc_prune_parts: the term limit over the union of several Hamiltonians
    (the partitions of one) on one device; returns the rows removed in all."""
    parts = list(parts)
    arr = (_vp * max(len(parts), 1))(*[H._h for H in parts])
    removed = ctypes.c_int64(0)
    st = _prune_parts(arr, len(parts), float(eps), int(max_terms), ctypes.byref(removed))
    if st != 0:
        msgs = [_err(H._h).decode() for H in parts if H._h]
        msg = next((m for m in msgs if m != "no error"), _err(None).decode())
        raise IqccError(st, msg)
    return removed.value


def iqcc_qmf_energy(H: Hamiltonian, theta, phi) -> float:
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    e = ctypes.c_double(0.0)
    H._check(_energy(H._h, tp, pp, ctypes.byref(e)))
    return e.value


def iqcc_generator_abc(H: Hamiltonian, gx, gz, theta, phi):
    gxa, gxp = _u64(gx, (H.W,))
    gza, gzp = _u64(gz, (H.W,))
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    out = np.zeros(3)
    H._check(_abc(H._h, gxp, gzp, tp, pp, out.ctypes.data_as(_f64p)))
    return out


def iqcc_energy_gradients(H: Hamiltonian, theta, phi, gx=None, gz=None, tau: float = 0.0):
    """(E(tau), dE/dtheta, dE/dphi, dE/dtau) after the generator (gx, gz) at
    amplitude tau; without a generator, the energy of H and its angle gradient."""
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    if (gx is None) != (gz is None):
        raise ValueError("gx and gz must be given together")
    gxp = gzp = None
    if gx is not None:
        gxa, gxp = _u64(gx, (H.W,))
        gza, gzp = _u64(gz, (H.W,))
    e = np.zeros(1)
    dt = np.zeros(H.n)
    dp = np.zeros(H.n)
    dtau = np.zeros(1)
    H._check(_egrad(H._h, gxp, gzp, float(tau), tp, pp, e.ctypes.data_as(_f64p), dt.ctypes.data_as(_f64p),
                    dp.ctypes.data_as(_f64p), dtau.ctypes.data_as(_f64p)))
    return float(e[0]), dt, dp, float(dtau[0])


def iqcc_dis_gradients(H: Hamiltonian, theta, phi, cx=None, cz=None, cap: int | None = None):
    """With candidates: their gradients.  Without: the ordered DIS (cx, cz, g),
    at most ``cap`` of them (all when cap is None)."""
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    n_out = ctypes.c_int64(0)
    if cx is not None:
        cxa, cxp = _u64(cx, (-1, H.W))
        cza, czp = _u64(cz, (-1, H.W))
        g = np.zeros(max(len(cxa), 1))
        H._check(_dis(H._h, tp, pp, len(cxa), cxp, czp, 0, ctypes.byref(n_out), None, None,
                      g.ctypes.data_as(_f64p)))
        return g[: len(cxa)]
    if cap is None:
        H._check(_dis(H._h, tp, pp, 0, None, None, 0, ctypes.byref(n_out), None, None, None))
        cap = n_out.value
    k = max(int(cap), 1)
    ox = np.zeros((k, H.W), np.uint64)
    oz = np.zeros((k, H.W), np.uint64)
    og = np.zeros(k)
    H._check(_dis(H._h, tp, pp, 0, None, None, int(cap), ctypes.byref(n_out), ox.ctypes.data_as(_u64p),
                  oz.ctypes.data_as(_u64p), og.ctypes.data_as(_f64p)))
    m = min(int(cap), n_out.value)
    return ox[:m], oz[:m], og[:m]


def iqcc_iterate(H: Hamiltonian, theta, phi, n_gen: int, eps: float = 0.0, max_terms: int = 0,
                 min_gradient: float = 0.0, forced_x=None, forced_z=None, forced_tau=None,
                 screening: int = 0) -> dict:
    ta, tp = _f64(theta, H.n)
    pa, pp = _f64(phi, H.n)
    keep = []
    o = iqcc_iter_opts(n_gen, eps, max_terms, min_gradient, 0, None, None, None, int(screening))
    if forced_x is not None:
        fxa, fxp = _u64(forced_x, (-1, H.W))
        fza, fzp = _u64(forced_z, (-1, H.W))
        keep += [fxa, fza]
        o.n_forced, o.forced_x, o.forced_z = len(fxa), fxp, fzp
        if forced_tau is not None:
            fta, ftp = _f64(forced_tau, len(fxa))
            keep.append(fta)
            o.forced_tau = ftp
    r = iqcc_iter_result()
    H._check(_iterate(H._h, tp, pp, ctypes.byref(o), ctypes.byref(r)))
    k, W = r.n_applied, H.W
    return {"gx": np.array(r.gx[: k * W], np.uint64).reshape(k, W),
            "gz": np.array(r.gz[: k * W], np.uint64).reshape(k, W),
            "g": np.array(r.grad[:k]), "tau": np.array(r.tau[:k]),
            "abc": np.array([list(r.abc[i]) for i in range(k)]).reshape(k, 3),
            "removed": r.n_removed, "energy": r.energy, "M": r.n_terms, "M_before": r.n_terms_before,
            "M_peak": r.n_terms_peak, "dressed_terms": r.dressed_terms}


def iqcc_num_terms(H: Hamiltonian) -> int:
    m = ctypes.c_int64(0)
    H._check(_num(H._h, ctypes.byref(m)))
    return m.value


def iqcc_export(H: Hamiltonian, out=None):
    """(x, z, c) in canonical order; ``out`` = preallocated (x, z, c) host arrays
    (e.g. pinned), filled in place."""
    n = ctypes.c_int64(0)
    H._check(_export(H._h, 0, ctypes.byref(n), None, None, None))
    m = n.value
    if out is None:
        x = np.zeros((max(m, 1), H.W), np.uint64)
        z = np.zeros((max(m, 1), H.W), np.uint64)
        c = np.zeros(max(m, 1))
    else:
        x, z, c = out
    H._check(_export(H._h, m, ctypes.byref(n), x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                     c.ctypes.data_as(_f64p)))
    return x[:m], z[:m], c[:m]


def iqcc_export_rows(H: Hamiltonian, out=None):
    """(x, z, c) in the context's storage order (iqcc_export_rows: no sort);
    ``out`` as for iqcc_export."""
    n = ctypes.c_int64(0)
    H._check(_export_rows(H._h, 0, ctypes.byref(n), None, None, None))
    m = n.value
    if out is None:
        x = np.zeros((max(m, 1), H.W), np.uint64)
        z = np.zeros((max(m, 1), H.W), np.uint64)
        c = np.zeros(max(m, 1))
    else:
        x, z, c = out
    H._check(_export_rows(H._h, m, ctypes.byref(n), x.ctypes.data_as(_u64p), z.ctypes.data_as(_u64p),
                          c.ctypes.data_as(_f64p)))
    return x[:m], z[:m], c[:m]


def iqcc_set_bin_slack(H: Hamiltonian, frac: float, rows: int) -> None:
    H._check(_bin_slack(H._h, float(frac), int(rows)))


def iqcc_get_stats(H: Hamiltonian) -> dict:
    s = iqcc_stats()
    H._check(_stats(H._h, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in iqcc_stats._fields_ if name != "pad"}


def iqcc_reset_stats(H: Hamiltonian) -> None:
    H._check(_reset(H._h))


def iqcc_set_wait_limit(H: Hamiltonian, polls: int) -> None:
    """Polls a device wait makes before it gives up with IQCC_ERR_TIMEOUT (0: the default)."""
    H._check(_set_wait(H._h, int(polls)))


def iqcc_wait_selftest(H: Hamiltonian) -> None:
    """One device wait on a word nothing writes: always raises IQCC_ERR_TIMEOUT."""
    H._check(_wait_selftest(H._h))


def iqcc_last_error(H: Hamiltonian | None = None) -> str:
    return _err(H._h if H is not None else None).decode()


def iqcc_free(H: Hamiltonian) -> None:
    H.close()


def exported_symbols():
    """Names of the C entry points this binding resolves."""
    return sorted(n for n in globals() if n.startswith("iqcc_") and callable(globals()[n]))


def iqcc_qmf_energy_noalloc(n_qubits: int, d_rows, d_coef, n_terms: int, theta, phi, stream=None) -> float:
    """QMF energy of rows already on the device, with no device allocation.

    ``d_rows`` / ``d_coef``: device addresses (ints) or CUDA tensors holding
    [n_terms][2*Wd] uint64 rows (x words then z words, Wd = 1, 2 or 4) and
    [n_terms] float64 coefficients.  ``stream``: a cudaStream_t handle, a
    torch stream, or None (then PyTorch's current stream when available)."""
    def addr(v):
        return int(v.data_ptr()) if hasattr(v, "data_ptr") else int(v)

    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            stream = None
    elif hasattr(stream, "cuda_stream"):
        stream = stream.cuda_stream
    ta, tp = _f64(theta, n_qubits)
    pa, pp = _f64(phi, n_qubits)
    e = ctypes.c_double(0.0)
    st = _energy_noalloc(int(n_qubits), int(n_terms), addr(d_rows), addr(d_coef), tp, pp, stream, ctypes.byref(e))
    if st != 0:
        raise IqccError(st, _err(None).decode())
    return e.value


# ---------------------------------------------------------------- batches of Hamiltonians

class iqcc_batch_screen_out(ctypes.Structure):
    _fields_ = [("energy", _f64p), ("gx", _u64p), ("gz", _u64p), ("grad", _f64p), ("abc", _f64p), ("tau", _f64p),
                ("n_terms", _i64p)]


class iqcc_batch_info(ctypes.Structure):
    _fields_ = [("n_terms", ctypes.c_int64), ("screens", ctypes.c_int64), ("graph_replays", ctypes.c_int64),
                ("blocks_energy", ctypes.c_int), ("blocks_group", ctypes.c_int), ("blocks_abc", ctypes.c_int),
                ("pad", ctypes.c_int)]


_bload = _sig("iqcc_batch_load", _c, [ctypes.POINTER(_vp), ctypes.POINTER(iqcc_opts), ctypes.c_int,
                                       ctypes.POINTER(ctypes.c_int), _i64p, _u64p, _u64p, _f64p])
_bscreen = _sig("iqcc_batch_screen", _c, [_vp, _f64p, _f64p, ctypes.POINTER(iqcc_batch_screen_out)])
_bstep = _sig("iqcc_batch_step", _c, [_vp, _f64p, _f64p, ctypes.c_double, ctypes.POINTER(iqcc_batch_screen_out),
                                       _f64p, _i64p])
_bexport = _sig("iqcc_batch_export", _c, [_vp, ctypes.c_int, ctypes.c_int64, _i64p, _u64p, _u64p, _f64p])
_binfo = _sig("iqcc_batch_get_info", _c, [_vp, ctypes.POINTER(iqcc_batch_info)])
_berr = _sig("iqcc_batch_last_error", ctypes.c_char_p, [_vp])
_bfree = _sig("iqcc_batch_free", None, [_vp])


class Batch:
    """Independent Hamiltonians of up to 48 qubits each, resident together (an ``iqcc_batch``)."""

    def __init__(self, handle, n_qubits, keepalive):
        self._h = handle
        self.n = list(n_qubits)
        self.B = len(self.n)
        self._keepalive = keepalive

    def _check(self, st):
        if st != 0:
            raise IqccError(st, _berr(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            _bfree(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def _angles(self, theta, phi):
        t = np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in theta])
        p = np.concatenate([np.asarray(a, np.float64).reshape(-1) for a in phi])
        if len(t) != sum(self.n) or len(p) != sum(self.n):
            raise ValueError("one angle per qubit of every problem")
        return _f64(t), _f64(p)


def _screen_out(B):
    arrs = {"energy": np.zeros(B), "gx": np.zeros(B, np.uint64), "gz": np.zeros(B, np.uint64),
            "grad": np.zeros(B), "abc": np.zeros((B, 3)), "tau": np.zeros(B), "n_terms": np.zeros(B, np.int64)}
    s = iqcc_batch_screen_out(arrs["energy"].ctypes.data_as(_f64p), arrs["gx"].ctypes.data_as(_u64p),
                              arrs["gz"].ctypes.data_as(_u64p), arrs["grad"].ctypes.data_as(_f64p),
                              arrs["abc"].ctypes.data_as(_f64p), arrs["tau"].ctypes.data_as(_f64p),
                              arrs["n_terms"].ctypes.data_as(_i64p))
    return arrs, s


def iqcc_batch_load(problems, capacity: int = 0, max_probe: int = 0, use_torch: bool = True,
                    device=None) -> Batch:
    """``problems``: a list of (n_qubits, x, z, coef) with one word per string."""
    n = [int(p[0]) for p in problems]
    xs = [np.asarray(p[1], np.uint64).reshape(-1) for p in problems]
    zs = [np.asarray(p[2], np.uint64).reshape(-1) for p in problems]
    cs = [np.asarray(p[3], np.float64).reshape(-1) for p in problems]
    offsets = np.zeros(len(problems) + 1, np.int64)
    offsets[1:] = np.cumsum([len(c) for c in cs])
    xa, xp = _u64(np.concatenate(xs) if xs else np.zeros(0, np.uint64))
    za, zp = _u64(np.concatenate(zs) if zs else np.zeros(0, np.uint64))
    ca, cp = _f64(np.concatenate(cs) if cs else np.zeros(0))
    na = (ctypes.c_int * len(n))(*n)
    stream, alloc, free = _torch_hooks(device, False) if use_torch else (None, None, None)
    opts = iqcc_opts(64, capacity, max_probe, stream, alloc or ALLOC_FN(), free or FREE_FN(), None)
    h = _vp()
    st = _bload(ctypes.byref(h), ctypes.byref(opts), len(n), na, offsets.ctypes.data_as(_i64p), xp, zp, cp)
    if st != 0:
        raise IqccError(st, _err(None).decode())
    return Batch(h, n, (alloc, free))


def iqcc_batch_screen(batch: Batch, theta, phi) -> dict:
    """Per problem: energy, best DIS candidate (gx, gz), its gradient, A, B, C, tau*, term count."""
    (ta, tp), (pa, pp) = batch._angles(theta, phi)
    arrs, s = _screen_out(batch.B)
    batch._check(_bscreen(batch._h, tp, pp, ctypes.byref(s)))
    return arrs


def iqcc_batch_step(batch: Batch, theta, phi, eps: float = 0.0):
    """Screen, dress every problem with its best candidate at tau*, prune eps:
    (screening dict, energies after, term counts after)."""
    (ta, tp), (pa, pp) = batch._angles(theta, phi)
    arrs, s = _screen_out(batch.B)
    ea = np.zeros(batch.B)
    na = np.zeros(batch.B, np.int64)
    batch._check(_bstep(batch._h, tp, pp, float(eps), ctypes.byref(s), ea.ctypes.data_as(_f64p),
                        na.ctypes.data_as(_i64p)))
    return arrs, ea, na


def iqcc_batch_export(batch: Batch, problem: int):
    n = ctypes.c_int64(0)
    batch._check(_bexport(batch._h, int(problem), 0, ctypes.byref(n), None, None, None))
    k = n.value
    x = np.zeros(k, np.uint64)
    z = np.zeros(k, np.uint64)
    c = np.zeros(k)
    batch._check(_bexport(batch._h, int(problem), k, ctypes.byref(n), x.ctypes.data_as(_u64p),
                          z.ctypes.data_as(_u64p), c.ctypes.data_as(_f64p)))
    return x.reshape(-1, 1), z.reshape(-1, 1), c


def iqcc_batch_get_info(batch: Batch) -> dict:
    s = iqcc_batch_info()
    batch._check(_binfo(batch._h, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in iqcc_batch_info._fields_ if name != "pad"}


def iqcc_batch_last_error(batch: Batch | None = None) -> str:
    return _berr(batch._h if batch is not None else None).decode()


def iqcc_batch_free(batch: Batch) -> None:
    batch.close()
