"""The synthetic-input generator against an independent construction (CPU).

The Jordan-Wigner Hamiltonian of seeded integrals (Eq. 1 -> Eq. 2) must equal,
as a dense matrix, the second-quantised Hamiltonian built directly in the
occupation-number basis with a+_P |n> = (-1)^{sum_{k<P} n_k} |n + e_P>.
"""
import numpy as np
import pytest

from paper_2603_08883_gb300 import synth
from tests import dense


def _fock_creators(n):
    """Dense a+_P in the basis index b, occupation n_j = bit (n-1-j) of b."""
    N = 2 ** n
    ops = []
    for P in range(n):
        A = np.zeros((N, N))
        for b in range(N):
            occ = [(b >> (n - 1 - j)) & 1 for j in range(n)]
            if occ[P]:
                continue
            sign = (-1) ** sum(occ[:P])
            b2 = b | (1 << (n - 1 - P))
            A[b2, b] = sign
        ops.append(A)
    return ops


def _fock_hamiltonian(h, eri):
    norb = h.shape[0]
    n = 2 * norb
    ad = _fock_creators(n)
    a = [m.T for m in ad]
    H = np.zeros((2 ** n, 2 ** n))
    for P in range(n):
        for Q in range(n):
            if P % 2 == Q % 2:
                H += h[P // 2, Q // 2] * ad[P] @ a[Q]
    for p in range(norb):
        for q in range(norb):
            for r in range(norb):
                for s in range(norb):
                    v = eri[p, q, r, s]
                    for sg in range(2):
                        for tg in range(2):
                            P, Q, R, S = 2 * p + sg, 2 * q + sg, 2 * r + tg, 2 * s + tg
                            H += 0.5 * v * ad[P] @ ad[R] @ a[S] @ a[Q]
    return H


@pytest.mark.parametrize("kind,norb,seed", [("plain", 2, 1), ("plain", 3, 8), ("decay", 3, 5), ("dblock", 3, 7)])
def test_jordan_wigner_matches_fock_space(kind, norb, seed):
    h, eri = synth.integrals(kind, norb, seed)
    n, x, z, c = synth.jordan_wigner(h, eri, rel_drop=0.0)
    assert n == 2 * norb
    Hj = dense.dense(n, x, z, c)
    Hf = _fock_hamiltonian(h, eri)
    assert np.abs(Hj - Hf).max() < 1e-12
    # real strings only: an even number of Y letters in every key
    ny = [bin(int(x[i, 0]) & int(z[i, 0])).count("1") for i in range(len(c))]
    assert all(v % 2 == 0 for v in ny)
    keys = np.concatenate([x, z], 1)
    assert len(np.unique(keys, axis=0)) == len(keys)


def test_integrals_have_eightfold_symmetry():
    for kind in ("plain", "decay", "dblock"):
        h, eri = synth.integrals(kind, 5, 3)
        assert np.array_equal(h, h.T)
        for perm in [(1, 0, 2, 3), (0, 1, 3, 2), (2, 3, 0, 1), (3, 2, 1, 0)]:
            assert np.array_equal(eri, eri.transpose(perm))


def test_workload_sizes():
    """The small workloads have the sizes their recipes give (regression pins
    of the generator, not of the method)."""
    n, x, z, c = synth.workload_hamiltonian(synth.WORKLOADS["jw8"])
    assert (n, len(c)) == (8, 361)
    n, x, z, c = synth.workload_hamiltonian(synth.WORKLOADS["jw24"])
    assert (n, len(c)) == (24, 29737)


def test_random_hamiltonian_edge_shapes():
    for n in (1, 63, 64, 65, 130, 200):
        _, x, z, c = synth.random_hamiltonian(n, 50, n)
        W = (n + 63) // 64
        assert x.shape[1] == W and z.shape[1] == W
        r = n - 64 * (W - 1)
        if r < 64:
            assert int((x[:, -1] >> np.uint64(r)).max()) == 0
            assert int((z[:, -1] >> np.uint64(r)).max()) == 0
        gx, gz = synth.random_generator(n, np.random.Generator(np.random.PCG64(n)))
        ny = sum(bin(int(a) & int(b)).count("1") for a, b in zip(gx, gz))
        assert ny % 2 == 1
