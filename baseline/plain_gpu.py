"""Plain PyTorch-tensor form of the iQCC dressing path, on the GPU.

This is the comparison that the library is timed against on the same GPU:
each step is written with stock tensor operations (bitwise ops, a SWAR
popcount, torch.unique over key rows, index_add_, gathers from small tables),
with no custom kernel.  It computes what the library computes:

* dress by one generator P at amplitude tau (Eq. 5, with the library's sign
  convention T -> cos(tau) T + sin(tau) iTP): every string T that anticommutes
  with P contributes cos(tau) c_T to itself and s_T sin(tau) c_T to its
  partner q = T xor P, where iTP = s_T P(q); equal keys are merged by summing
  their contributions (torch.unique over key rows, then index_add_);
* pruning of |c| < eps, and a term limit that keeps the largest |c| (ties at
  the threshold broken by torch.topk, not by key order);
* the QMF energy E = sum_T c_T prod_j beta_j(T_j) (Eq. 3, Eq. 12), with
  per-nibble tables of the product of four qubit factors;
* A, B, C of E(tau) = A + B cos(tau) + C sin(tau) for a generator.

Keys are int64 rows [M, 2W] (x words, then z words) holding the uint64 bits
of the symplectic encoding; coefficients are float64.  It runs wherever its
tensors live; bench.py gives it the GPU.
"""
import math

import numpy as np
import torch


def _i64(v: int) -> int:
    return v - (1 << 64) if v >= (1 << 63) else v


_M1 = _i64(0x5555555555555555)
_M2 = _i64(0x3333333333333333)
_M4 = _i64(0x0F0F0F0F0F0F0F0F)


def popcount(t: torch.Tensor) -> torch.Tensor:
    """Bits set in each int64 element (SWAR; the arithmetic right shifts only
    bring in bits that the masks clear)."""
    t = t - ((t >> 1) & _M1)
    t = (t & _M2) + ((t >> 2) & _M2)
    t = (t + (t >> 4)) & _M4
    t = t + (t >> 8)
    t = t + (t >> 16)
    t = t + (t >> 32)
    return t & 0x7F


def _as_i64(a, device) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint64).view(np.int64)).to(device)


class PlainHamiltonian:
    """H = sum_T c_T T as key rows and coefficients on `device`."""

    def __init__(self, n_qubits: int, x, z, coef, device="cuda"):
        self.n = n_qubits
        self.W = (n_qubits + 63) // 64
        self.device = torch.device(device)
        x = np.asarray(x, np.uint64).reshape(-1, self.W)
        z = np.asarray(z, np.uint64).reshape(-1, self.W)
        keys = torch.cat([_as_i64(x, self.device), _as_i64(z, self.device)], 1)
        c = torch.from_numpy(np.asarray(coef, np.float64)).to(self.device)
        self.keys, self.c = self._merge(keys, c)
        nz = self.c != 0
        self.keys, self.c = self.keys[nz], self.c[nz]

    def __len__(self) -> int:
        return int(self.c.shape[0])

    @staticmethod
    def _merge(keys, vals):
        uniq, inv = torch.unique(keys, dim=0, return_inverse=True)
        out = torch.zeros(uniq.shape[0], dtype=vals.dtype, device=vals.device)
        out.index_add_(0, inv, vals)
        return uniq, out

    def _gen(self, gx, gz):
        px = _as_i64(np.asarray(gx, np.uint64).reshape(self.W), self.device)
        pz = _as_i64(np.asarray(gz, np.uint64).reshape(self.W), self.device)
        return px, pz

    def _classify(self, px, pz):
        """Anticommuting mask, partner keys and the signs s_T of iTP = s_T P(q)."""
        W = self.W
        x, z = self.keys[:, :W], self.keys[:, W:]
        anti = (popcount((x & pz) ^ (z & px)).sum(1) & 1).bool()
        xa, za = x[anti], z[anti]
        qx, qz = xa ^ px, za ^ pz
        # i^{|x_T & z_T|} X^{x_T} Z^{z_T} times i^{|x_P & z_P|} X^{x_P} Z^{z_P}: moving Z^{z_T} past X^{x_P}
        # gives (-1)^{|z_T & x_P|}; the product is i^e P(q) with e as below, and iTP = i^{e+1} P(q)
        e = (popcount(xa & za).sum(1) + int(popcount(px & pz).sum()) + 2 * popcount(za & px).sum(1)
             - popcount(qx & qz).sum(1)) % 4
        s = torch.where(e == 3, 1.0, -1.0).to(torch.float64)
        return anti, torch.cat([qx, qz], 1), s

    def dress(self, gx, gz, tau: float) -> None:
        px, pz = self._gen(gx, gz)
        anti, q, s = self._classify(px, pz)
        ct, st = math.cos(tau), math.sin(tau)
        vals = torch.cat([torch.where(anti, self.c * ct, self.c), s * self.c[anti] * st])
        self.keys, self.c = self._merge(torch.cat([self.keys, q]), vals)

    def prune(self, eps: float, max_terms: int = 0) -> int:
        m0 = len(self)
        keep = self.c.abs() >= eps
        self.keys, self.c = self.keys[keep], self.c[keep]
        if max_terms > 0 and len(self) > max_terms:
            idx = torch.topk(self.c.abs(), max_terms, sorted=False).indices
            self.keys, self.c = self.keys[idx], self.c[idx]
        return m0 - len(self)

    def _nibble_tables(self, theta, phi):
        """Per group of 4 qubits, the product of their factors for each of the 256 (x, z) nibble pairs."""
        th = np.asarray(theta, np.float64)
        ph = np.asarray(phi, np.float64)
        groups = (self.n + 3) // 4
        tab = np.ones((groups, 256))
        for g in range(groups):
            for code in range(256):
                xb, zb = code & 15, code >> 4
                v = 1.0
                for k in range(4):
                    j = 4 * g + k
                    if j >= self.n:
                        continue
                    bx, bz = (xb >> k) & 1, (zb >> k) & 1
                    if bx and bz:
                        v *= math.sin(th[j]) * math.sin(ph[j])
                    elif bx:
                        v *= math.sin(th[j]) * math.cos(ph[j])
                    elif bz:
                        v *= math.cos(th[j])
                tab[g, code] = v
        return torch.from_numpy(tab).to(self.device)

    def _expect(self, keys, tab):
        """<Omega|T|Omega> of every key row."""
        W = self.W
        out = torch.ones(keys.shape[0], dtype=torch.float64, device=self.device)
        for g in range(tab.shape[0]):
            w, sh = divmod(4 * g, 64)
            xb = (keys[:, w] >> sh) & 15
            zb = (keys[:, W + w] >> sh) & 15
            out = out * tab[g][xb | (zb << 4)]
        return out

    def energy(self, theta, phi) -> float:
        return float((self.c * self._expect(self.keys, self._nibble_tables(theta, phi))).sum())

    def abc(self, gx, gz, theta, phi):
        tab = self._nibble_tables(theta, phi)
        px, pz = self._gen(gx, gz)
        anti, q, s = self._classify(px, pz)
        ev = self._expect(self.keys, tab)
        a = float((self.c[~anti] * ev[~anti]).sum())
        b = float((self.c[anti] * ev[anti]).sum())
        cc = float((s * self.c[anti] * self._expect(q, tab)).sum())
        return a, b, cc

    def export(self):
        """(x, z, c) as host arrays in canonical order (x as an integer with the
        last word most significant, then z likewise)."""
        keys = self.keys.cpu().numpy().view(np.uint64)
        c = self.c.cpu().numpy()
        W = self.W
        order = np.lexsort([keys[:, W + w] for w in range(W)] + [keys[:, w] for w in range(W)])
        return keys[order, :W].copy(), keys[order, W:].copy(), c[order].copy()
