"""Sort-based dressing (iqcc_dress_sorted: expansion, radix sort, segmented
sum) against the oracle and against the hash path of iqcc_dress."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests.compare import compare

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)


def _gens(n, rng, k, weight=None):
    gens = [synth.random_generator(n, rng, weight) for _ in range(k)]
    return np.array([g[0] for g in gens]), np.array([g[1] for g in gens]), rng.uniform(-math.pi, math.pi, k)


@pytest.mark.parametrize("n,m", [(1, 3), (7, 90), (24, 4000), (64, 6000), (65, 6000), (100, 20_000), (130, 5000),
                                 (200, 3000)])
@pytest.mark.parametrize("fuse", [1, 3])
def test_sorted_dress_matches_oracle(n, m, fuse):
    rng = np.random.Generator(np.random.PCG64(17 * n + fuse))
    _, x, z, c = synth.random_hamiltonian(n, m, 4000 + n)
    gx, gz, taus = _gens(n, rng, 4)
    o = oracle.Oracle(n, x, z, c)
    for k in range(4):
        o.dress(gx[k], gz[k], taus[k])
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    assert iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=fuse) == 4
    scale = float(np.abs(c).max())
    bad = compare(iqcc.iqcc_export(H), o.export(), scale=scale)
    assert not bad, bad[:5]
    s = iqcc.iqcc_get_stats(H)
    assert s["n_sorted_groups"] == (4 + fuse - 1) // fuse


@pytest.mark.parametrize("n", [20, 100])
def test_sorted_and_hash_dress_agree(n):
    """Same input, same generators: the two merges give the same Hamiltonian up
    to rounding, the same key set, and the index is usable afterwards."""
    rng = np.random.Generator(np.random.PCG64(n))
    _, x, z, c = synth.random_hamiltonian(n, 30_000, 600 + n)
    gx, gz, taus = _gens(n, rng, 3)
    Ha = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    Hb = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_dress(Ha, gx, gz, taus)
    iqcc.iqcc_dress_sorted(Hb, gx, gz, taus)
    assert len(Ha) == len(Hb)
    assert not compare(iqcc.iqcc_export(Hb), iqcc.iqcc_export(Ha), scale=float(np.abs(c).max()))
    # index rebuilt: a further hash dress and the energy still match the oracle
    o = oracle.Oracle(n, x, z, c)
    for k in range(3):
        o.dress(gx[k], gz[k], taus[k])
    g2x, g2z, t2 = _gens(n, rng, 1)
    iqcc.iqcc_dress(Hb, g2x, g2z, t2)
    o.dress(g2x[0], g2z[0], t2[0])
    assert not compare(iqcc.iqcc_export(Hb), o.export(), scale=float(np.abs(c).max()))
    th, ph = synth.qmf_angles(n, "uniform", seed=3)
    assert iqcc.iqcc_qmf_energy(Hb, th, ph) == pytest.approx(o.energy(th, ph), abs=1e-9)


def test_sorted_dress_keeps_exact_zeros_and_reports_capacity():
    n = 6
    x = np.array([[0b000001]], np.uint64)   # X0
    z = np.zeros((1, 1), np.uint64)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, np.array([1.0]))
    P = (np.array([[0b1]], np.uint64), np.array([[0b1]], np.uint64))  # Y0 anticommutes with X0
    iqcc.iqcc_dress_sorted(H, P[0], P[1], [0.0])          # partner appended with coefficient 0
    Hh = iqcc.iqcc_load_hamiltonian(n, x, z, np.array([1.0]))
    iqcc.iqcc_dress(Hh, P[0], P[1], [0.0])
    assert len(H) == len(Hh) == 2
    # capacity: a group that would expand past it fails and leaves H unchanged
    _, x, z, c = synth.random_hamiltonian(40, 3000, 9)
    H = iqcc.iqcc_load_hamiltonian(40, x, z, c, capacity=3100)
    before = iqcc.iqcc_export(H)
    rng = np.random.Generator(np.random.PCG64(1))
    gx, gz, taus = _gens(40, rng, 6, weight=1)
    with pytest.raises(iqcc.IqccError) as err:
        iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=6)
    assert err.value.status == 4
    after = iqcc.iqcc_export(H)
    assert all(np.array_equal(a, b) for a, b in zip(before, after))
    with pytest.raises(iqcc.IqccError) as err:
        iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=9)
    assert err.value.status == 1


def test_sorted_dress_fused_iteration_24_qubits():
    """The four generators of an iteration of the 24-qubit workload fused into
    one expansion and one sort, against the oracle's sequential dress."""
    w = synth.WORKLOADS["jw24"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    o = oracle.Oracle(n, x, z, c)
    res = o.iterate(th, ph, w.n_gen, 0.0, 0)
    gx, gz, taus = res["gx"], res["gz"], res["tau"]
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    assert iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=w.n_gen) == w.n_gen
    assert not compare(iqcc.iqcc_export(H), o.export(), scale=float(np.abs(c).max()))
