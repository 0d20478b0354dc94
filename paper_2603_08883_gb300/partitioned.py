"""Partitioned Hamiltonians: H split by key bits over several contexts (App. B).

A partition is the set of strings that share the values of chosen key bits
(``mx`` / ``mz``: masks over the x and z words).  A generator P whose masked
bits are zero keeps each anticommuting row and its partner T xor P in the same
partition, so each part is dressed on its own.  Otherwise every anticommuting
row of partition a has its partner in partition a xor shift(P).

``PartitionedHamiltonian`` keeps the parts as separate contexts on one GPU and
runs every step in the library: a crossing generator dresses each pair of
partitions together (``iqcc_dress_pair``: both parts' anticommuting rows in
one set of pair bins, every output row to the partition owning its key), A, B,
C and the energy are summed over the parts (``iqcc_generator_abc_parts``), and
the term limit is taken over all parts on the device (``iqcc_prune_parts``).

``exchange_dress`` and ``reduced_tau`` are the steps for one part per process
(a multi-process layout, not built for GPUs here): each side sends its
anticommuting rows (``iqcc_cross_rows``) and applies the dress to its own rows
with the other side's (``iqcc_dress_cross``), moving rows with
torch.distributed; the engine is anything with the four methods of
``ContextEngine``.
"""
from __future__ import annotations

import math

import numpy as np


def _lib():
    from . import iqcc  # the CUDA library: loaded only by the parts that run on the device
    return iqcc


def _mask_bits(mx, mz, W: int):
    """(word, bit, is_z) of every set bit of the masks, x words first."""
    out = []
    for which, m in ((0, mx), (1, mz)):
        m = np.asarray(m, np.uint64).reshape(W)
        for w in range(W):
            v = int(m[w])
            while v:
                b = (v & -v).bit_length() - 1
                out.append((w, b, which))
                v &= v - 1
    return out


def partition_of(x, z, mx, mz) -> np.ndarray:
    """Partition index of each key (x, z: [M, W]): its masked bits, packed in mask order."""
    x = np.asarray(x, np.uint64)
    z = np.asarray(z, np.uint64)
    W = x.shape[1]
    part = np.zeros(x.shape[0], np.int64)
    for k, (w, b, which) in enumerate(_mask_bits(mx, mz, W)):
        col = (z if which else x)[:, w]
        part |= ((col >> np.uint64(b)) & np.uint64(1)).astype(np.int64) << k
    return part


def generator_shift(gx, gz, mx, mz) -> int:
    """Partition offset of P: the partner of a row of partition a lies in a xor shift."""
    return int(partition_of(np.asarray(gx, np.uint64).reshape(1, -1), np.asarray(gz, np.uint64).reshape(1, -1),
                            mx, mz)[0])


def closed_form_tau(a: float, b: float, c: float) -> float:
    """Minimiser of E(tau) = A + B cos(tau) + C sin(tau) (0 when B = C = 0)."""
    return 0.0 if (b == 0.0 and c == 0.0) else math.atan2(-c, -b)


class ContextEngine:
    """One partition held by a library context: the four steps the exchange needs."""

    def __init__(self, H):
        self.H = H

    def cross_rows(self, gx, gz):
        return _lib().iqcc_cross_rows(self.H, gx, gz)

    def dress_cross(self, gx, gz, tau, px, pz, pc):
        _lib().iqcc_dress_cross(self.H, gx, gz, tau, px, pz, pc)

    def dress(self, gx, gz, tau):
        _lib().iqcc_dress(self.H, np.asarray(gx).reshape(1, -1), np.asarray(gz).reshape(1, -1), [tau])

    def abc(self, gx, gz, theta, phi):
        return _lib().iqcc_generator_abc(self.H, gx, gz, theta, phi)


class PartitionedHamiltonian:
    """H split over 2^m contexts on this GPU by the m set bits of (mx, mz)."""

    def __init__(self, n_qubits: int, x, z, coef, mx, mz, **load_kwargs):
        self.n = n_qubits
        self.W = (n_qubits + 63) // 64
        self.mx = np.asarray(mx, np.uint64).reshape(self.W)
        self.mz = np.asarray(mz, np.uint64).reshape(self.W)
        m = len(_mask_bits(self.mx, self.mz, self.W))
        x = np.asarray(x, np.uint64).reshape(-1, self.W)
        z = np.asarray(z, np.uint64).reshape(-1, self.W)
        coef = np.asarray(coef, np.float64)
        part = partition_of(x, z, self.mx, self.mz)
        self.parts = []
        for a in range(1 << m):
            sel = part == a
            self.parts.append(_lib().iqcc_load_hamiltonian(n_qubits, x[sel], z[sel], coef[sel], **load_kwargs))

    def __len__(self) -> int:
        return sum(len(H) for H in self.parts)

    def energy(self, theta, phi) -> float:
        zero = np.zeros(self.W, np.uint64)
        return _lib().iqcc_generator_abc_parts(self.parts, zero, zero, theta, phi)[0][0]

    def abc(self, gx, gz, theta, phi):
        return _lib().iqcc_generator_abc_parts(self.parts, gx, gz, theta, phi)[0]

    def pattern(self, a: int):
        """Key bits (x words, z words) of partition a under the masks."""
        px = np.zeros(self.W, np.uint64)
        pz = np.zeros(self.W, np.uint64)
        for k, (w, b, which) in enumerate(_mask_bits(self.mx, self.mz, self.W)):
            if (a >> k) & 1:
                (pz if which else px)[w] |= np.uint64(1) << np.uint64(b)
        return px, pz

    def dress(self, gx, gz, tau: float) -> None:
        """One generator: inside each part when P flips no partition bit, else
        over each pair of partitions (a, a xor shift) on the device
        (iqcc_dress_pair: one set of pair bins for both, every output row to
        the partition owning its key)."""
        d = generator_shift(gx, gz, self.mx, self.mz)
        if d == 0:
            for H in self.parts:
                ContextEngine(H).dress(gx, gz, tau)
            return
        for a in range(len(self.parts)):
            if a < a ^ d:
                ax, az = self.pattern(a)
                _lib().iqcc_dress_pair(self.parts[a], self.parts[a ^ d], gx, gz, tau, self.mx, self.mz, ax, az)

    def step(self, gx, gz, theta, phi) -> float:
        """The closed-form amplitude from the A, B, C summed over the parts, then the dress; returns tau."""
        _, tau = _lib().iqcc_generator_abc_parts(self.parts, gx, gz, theta, phi)
        self.dress(gx, gz, tau)
        return tau

    def prune(self, eps: float, max_terms: int = 0) -> int:
        """|C| < eps dropped in every part; with a term limit, the max_terms
        largest |C| of the whole Hamiltonian kept, ties at the threshold in
        canonical key order across the parts (iqcc_prune_parts: the threshold
        is found on the device over all parts)."""
        return _lib().iqcc_prune_parts(self.parts, eps, max_terms)

    def export(self):
        """All parts in canonical order (x as an integer, last word most significant, then z)."""
        xs, zs, cs = zip(*(_lib().iqcc_export(H) for H in self.parts))
        x, z, c = np.concatenate(xs), np.concatenate(zs), np.concatenate(cs)
        order = np.lexsort([z[:, w] for w in range(self.W)] + [x[:, w] for w in range(self.W)])
        return x[order], z[order], c[order]

    def close(self) -> None:
        for H in self.parts:
            H.close()
        self.parts = []


def _send_recv(dist, peer: int, arrays):
    """Send `arrays` (host numpy) to peer and receive the peer's arrays of the
    same dtypes and trailing shapes (the row count first)."""
    import torch
    k = np.array([arrays[0].shape[0]], np.int64)
    kin = torch.zeros(1, dtype=torch.int64)
    req = dist.isend(torch.from_numpy(k), peer)
    dist.recv(kin, peer)
    req.wait()
    n_in = int(kin[0])
    n_out = int(k[0])
    out = []
    for a in arrays:  # empty messages are skipped on both sides (each knows both counts)
        width = int(np.prod(a.shape[1:])) if a.ndim > 1 else 1
        flat = np.ascontiguousarray(a).reshape(a.shape[0], width)
        as_i64 = flat.view(np.int64) if flat.dtype == np.uint64 else flat
        buf = torch.zeros((n_in, flat.shape[1]), dtype=torch.from_numpy(as_i64[:0]).dtype)
        req = dist.isend(torch.from_numpy(np.ascontiguousarray(as_i64)), peer) if n_out else None
        if n_in:
            dist.recv(buf, peer)
        if req is not None:
            req.wait()
        got = buf.numpy()
        got = got.view(np.uint64) if flat.dtype == np.uint64 else got
        out.append(got.reshape((n_in,) + a.shape[1:]))
    return out


def reduced_tau(engine, dist, gx, gz, theta, phi) -> float:
    """Closed-form amplitude from this part's A, B, C summed over all ranks."""
    import torch
    s = torch.tensor(np.asarray(engine.abc(gx, gz, theta, phi), np.float64))
    dist.all_reduce(s)
    return closed_form_tau(*(float(v) for v in s))


def exchange_dress(engine, dist, rank: int, gx, gz, tau: float, mx, mz) -> None:
    """The dress of one part held by this rank (rank = partition index): local
    when P keeps pairs inside the partition, else one exchange with the rank
    that holds the partner partition."""
    d = generator_shift(gx, gz, mx, mz)
    if d == 0:
        engine.dress(gx, gz, tau)
        return
    px, pz, pc = _send_recv(dist, rank ^ d, list(engine.cross_rows(gx, gz)))
    engine.dress_cross(gx, gz, tau, px, pz, pc)
