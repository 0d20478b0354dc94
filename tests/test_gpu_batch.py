"""Batches of independent Hamiltonians (iqcc_batch_*): per-problem screening,
dress and compression against one oracle per problem, graph replay, errors."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests.compare import compare

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)


def _problems(seed=0):
    """Uneven problems: Jordan-Wigner molecules of 12-20 qubits and random
    Hamiltonians up to 48 qubits, plus one without any flip set."""
    out = []
    for k, norb in enumerate([6, 7, 8, 10]):
        h, eri = synth.integrals("decay", norb, 1000 + k + seed)
        n, x, z, c = synth.jordan_wigner(h, eri)
        out.append((n, x.reshape(-1), z.reshape(-1), c))
    for k, (n, m) in enumerate([(30, 4000), (48, 2500), (9, 300)]):
        _, x, z, c = synth.random_hamiltonian(n, m, 2000 + k + seed, density=0.3)
        x[: len(x) // 5] = 0  # diagonal strings for the energies
        out.append((n, x.reshape(-1), z.reshape(-1), c))
    z = np.arange(1, 40, dtype=np.uint64)
    out.append((6, np.zeros_like(z), z & np.uint64(63), np.linspace(-1, 1, len(z))))  # diagonal only
    return out


def _basis(n, filled=None):
    filled = n // 2 if filled is None else filled
    return np.where(np.arange(n) < filled, np.pi, 0.0), np.zeros(n)


def _oracle_check(o, n, th, ph, res, p, scale):
    """The GPU's screening of problem p against the oracle (the candidate must
    be a top choice; its gradient, A, B, C and tau* must match)."""
    assert res["energy"][p] == pytest.approx(o.energy(th, ph), abs=1e-9 * scale)
    cx, cz, g = o.dis(th, ph)
    if len(g) == 0:
        assert res["gx"][p] == 0 and res["tau"][p] == 0.0
        return None
    gx = np.array([res["gx"][p]], np.uint64)
    gz = np.array([res["gz"][p]], np.uint64)
    assert res["gx"][p] != 0
    g_o = o.gradient(gx, gz, th, ph)
    assert res["grad"][p] == pytest.approx(g_o, rel=1e-9, abs=1e-12 * scale)
    assert abs(g_o) >= np.max(np.abs(g)) * (1 - 1e-9) - 1e-12 * scale
    a, b, c = o.abc(gx, gz, th, ph)
    assert np.allclose(res["abc"][p], [a, b, c], rtol=1e-9, atol=1e-12 * scale)
    tau = 0.0 if (b == 0 and c == 0) else math.atan2(-c, -b)
    # the same rotation: tau = pi and -pi differ only in the sign of a zero C
    assert math.cos(res["tau"][p]) == pytest.approx(math.cos(tau), abs=1e-9)
    assert math.sin(res["tau"][p]) == pytest.approx(math.sin(tau), abs=1e-9)
    return gx, gz, tau


def test_batch_steps_match_one_oracle_per_problem():
    probs = _problems()
    B = len(probs)
    batch = iqcc.iqcc_batch_load(probs)
    orcs = [oracle.Oracle(n, x.reshape(-1, 1), z.reshape(-1, 1), c) for n, x, z, c in probs]
    angles = [_basis(n) for n, *_ in probs]
    th = [a[0] for a in angles]
    ph = [a[1] for a in angles]
    eps = 1e-10
    for step in range(3):
        res, e_after, n_after = iqcc.iqcc_batch_step(batch, th, ph, eps)
        for p, (n, x, z, c) in enumerate(probs):
            o = orcs[p]
            scale = float(np.abs(c).sum())
            assert res["n_terms"][p] == len(o)
            chosen = _oracle_check(o, n, th[p], ph[p], res, p, scale)
            if chosen is not None:
                o.dress(chosen[0], chosen[1], res["tau"][p])   # teacher-forced: the GPU's candidate and tau
            o.prune(eps, 0)
            assert n_after[p] == len(o)
            assert e_after[p] == pytest.approx(o.energy(th[p], ph[p]), abs=1e-9 * scale)
            bad = compare(iqcc.iqcc_batch_export(batch, p), o.export(), eps=eps, scale=float(np.abs(c).max()))
            assert not bad, (step, p, bad[:3])
    info = iqcc.iqcc_batch_get_info(batch)
    assert info["blocks_energy"] > 0 and info["blocks_group"] > 0 and info["blocks_abc"] > 0


def test_batch_screen_replays_its_graph_with_new_angles():
    probs = _problems(seed=7)
    batch = iqcc.iqcc_batch_load(probs)
    orcs = [oracle.Oracle(n, x.reshape(-1, 1), z.reshape(-1, 1), c) for n, x, z, c in probs]
    for k, filled in enumerate([None, 1, 0, 3]):
        angles = [_basis(n, None if filled is None else min(filled, n)) for n, *_ in probs]
        th = [a[0] for a in angles]
        ph = [a[1] for a in angles]
        res = iqcc.iqcc_batch_screen(batch, th, ph)
        for p, (n, x, z, c) in enumerate(probs):
            _oracle_check(orcs[p], n, th[p], ph[p], res, p, float(np.abs(c).sum()))
    info = iqcc.iqcc_batch_get_info(batch)
    assert info["screens"] == 4 and info["graph_replays"] == 3


def test_batch_errors():
    probs = _problems()
    with pytest.raises(iqcc.IqccError) as err:
        iqcc.iqcc_batch_load([(50, np.zeros(1, np.uint64), np.zeros(1, np.uint64), np.ones(1))])
    assert err.value.status == 1
    with pytest.raises(iqcc.IqccError) as err:  # a bit above the problem's qubit count
        iqcc.iqcc_batch_load([(4, np.array([16], np.uint64), np.zeros(1, np.uint64), np.ones(1))])
    assert err.value.status == 1
    batch = iqcc.iqcc_batch_load(probs)
    th = [np.full(n, 0.3) for n, *_ in probs]
    ph = [np.zeros(n) for n, *_ in probs]
    with pytest.raises(iqcc.IqccError) as err:   # not a z-eigenstate
        iqcc.iqcc_batch_screen(batch, th, ph)
    assert err.value.status == 1
    small = iqcc.iqcc_batch_load(probs[:1], capacity=len(probs[0][3]) + 10)
    th0, ph0 = _basis(probs[0][0])
    with pytest.raises(iqcc.IqccError) as err:   # no room for a dress
        iqcc.iqcc_batch_step(small, [th0], [ph0])
    assert err.value.status == 4
