"""GPU parity on the workload recipes, generator by generator.

An iteration (App. A steps 1-5) is driven through the C ABI one step at a
time, teacher-forced with the oracle's screening and amplitudes: DIS
gradients, then for each of the top generators A, B, C, the dress, and the
term limit after the dress (the cut to the max_terms largest |C|), then the
compression by eps and the energy.  After every dress and every cut the GPU's
Hamiltonian is compared with the oracle's: the key sets must be equal except
for keys within 1e-12 relative of that cut's threshold |C| (a tie up to
rounding, kept on one side and dropped on the other), and coefficients agree
to 1e-12 relative.  When such a key differs, the GPU is given the oracle's
Hamiltonian before the next step, so the difference does not propagate
(teacher forcing of H).  The same iteration is then run by iqcc_iterate with
the oracle's generators and amplitudes, from the oracle's Hamiltonian at the
start of the iteration, and compared with the oracle's end state.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests.compare import compare, cut_threshold

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)

E_TOL = 1e-9       # Ha


def _check_dis(H, o, th, ph, n_gen):
    """Oracle's DIS list against the GPU's: same candidates, gradients to 1e-12
    relative; the GPU's own top n_gen equal the oracle's up to |g| ties."""
    ox, oz, og = o.dis(th, ph)
    gx, gz, gg = iqcc.iqcc_dis_gradients(H, th, ph)
    assert len(gg) == len(og)
    ref = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(ox, oz, og)}
    got = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(gx, gz, gg)}
    assert ref.keys() == got.keys()
    scale = float(np.max(np.abs(og))) if len(og) else 0.0
    for k, v in ref.items():
        assert abs(got[k] - v) <= 1e-12 * abs(v) + 1e-14 * scale, (got[k], v)
    k = min(n_gen, len(og))
    if k:
        mag = np.abs(og)
        cut = mag[k - 1]
        sure = {(ox[i].tobytes(), oz[i].tobytes()) for i in range(k) if mag[i] > cut * (1 + 1e-9)}
        top = {(gx[i].tobytes(), gz[i].tobytes()) for i in range(k)}
        assert sure <= top
    return ox, oz, og


def _reload(H, o, n, capacity):
    x, z, c = o.export()
    H.close()
    return iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=capacity)


def iteration_by_steps(H, o, n, th, ph, n_gen, eps, cap, capacity):
    """One teacher-forced iteration step by step; returns (H, generators,
    amplitudes, number of cuts with a near-threshold key difference)."""
    ox, oz, og = _check_dis(H, o, th, ph, n_gen)
    sel = [i for i in range(len(og)) if abs(og[i]) > 1e-12][:n_gen]
    gens, taus, resyncs = [], [], 0
    for i in sel:
        P = (ox[i], oz[i])
        a_o = o.abc(*P, th, ph)
        a_g = iqcc.iqcc_generator_abc(H, *P, th, ph)
        assert np.allclose(a_g, a_o, rtol=0, atol=E_TOL), (a_g, a_o)
        tau = 0.0 if (a_o[1] == 0.0 and a_o[2] == 0.0) else math.atan2(-a_o[2], -a_o[1])
        o.dress(*P, tau)
        iqcc.iqcc_dress(H, P[0], P[1], [tau])
        gens.append(P)
        taus.append(tau)
        bad = compare(iqcc.iqcc_export(H), o.export())
        assert not bad, bad[:5]
        if cap > 0 and len(o) > cap:
            thr = cut_threshold(o.export()[2], cap)
            r_o = o.prune(0.0, cap)
            r_g = iqcc.iqcc_prune(H, 0.0, cap)
            assert len(H) == len(o) == cap
            assert r_g == r_o
            gpu, ref = iqcc.iqcc_export(H), o.export()
            bad = compare(gpu, ref, thresholds=[thr])
            assert not bad, bad[:5]
            if not np.array_equal(gpu[0], ref[0]) or not np.array_equal(gpu[1], ref[1]):
                resyncs += 1
                H = _reload(H, o, n, capacity)
    thr = cut_threshold(o.export()[2], cap) if cap > 0 and len(o) > cap else 0.0
    r_o = o.prune(eps, cap)
    r_g = iqcc.iqcc_prune(H, eps, cap)
    gpu, ref = iqcc.iqcc_export(H), o.export()
    bad = compare(gpu, ref, eps=eps, thresholds=[thr] if thr else ())
    assert not bad, bad[:5]
    if np.array_equal(gpu[0], ref[0]) and np.array_equal(gpu[1], ref[1]):
        assert r_g == r_o
    assert iqcc.iqcc_qmf_energy(H, th, ph) == pytest.approx(o.energy(th, ph), abs=E_TOL)
    return H, gens, taus, resyncs


def _run_recipe(n, x, z, c, th, ph, n_iter, n_gen, eps, cap):
    capacity = 2 * cap if cap > 0 else 0
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=capacity)
    cuts_seen = 0
    for it in range(n_iter):
        start = o.export()
        H, gens, taus, resyncs = iteration_by_steps(H, o, n, th, ph, n_gen, eps, cap, capacity)
        cuts_seen += 1 if cap > 0 and len(o) == cap else 0
        # the whole iteration through iqcc_iterate, from the same start, forced
        Hi = iqcc.iqcc_load_hamiltonian(n, *start, capacity=capacity)
        r = iqcc.iqcc_iterate(Hi, th, ph, n_gen, eps, cap, forced_x=np.array([g[0] for g in gens]),
                              forced_z=np.array([g[1] for g in gens]), forced_tau=np.array(taus))
        assert r["energy"] == pytest.approx(o.energy(th, ph), abs=E_TOL)
        if resyncs == 0:
            bad = compare(iqcc.iqcc_export(Hi), o.export(), eps=eps)
            assert not bad, bad[:5]
        Hi.close()
    return cuts_seen


def test_jw100_recipe_teacher_forced_with_term_limit():
    """The 100-qubit d-block recipe (50 orbitals, 8 generators per iteration,
    eps = 1e-8, basis reference), on its 2 x 10^5 largest strings with the term
    limit lowered to 3 x 10^5 so that the cut after every dress, the
    compaction and the growth of the row store all run; two iterations."""
    w = synth.WORKLOADS["jw100"]
    n, x, z, c = synth.workload_hamiltonian(w)
    keep = np.sort(np.argsort(-np.abs(c), kind="stable")[:200_000])
    th, ph = synth.workload_angles(w)
    cuts = _run_recipe(n, x[keep], z[keep], c[keep], th, ph, 2, w.n_gen, w.eps, 300_000)
    assert cuts >= 1


def test_jw24_recipe_term_limit_after_every_dress():
    """The 24-qubit recipe with a term limit of 60,000 (the cut after every
    dress from the first iteration on), three iterations."""
    w = synth.WORKLOADS["jw24"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    cuts = _run_recipe(n, x, z, c, th, ph, 3, w.n_gen, w.eps, 60_000)
    assert cuts >= 1


def test_jw24_recipe_without_term_limit():
    """The 24-qubit recipe as configured (no term limit, eps = 1e-10)."""
    w = synth.WORKLOADS["jw24"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    _run_recipe(n, x, z, c, th, ph, 3, w.n_gen, w.eps, 0)
