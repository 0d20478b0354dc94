"""Pins of the CPU oracle against things other than itself (CPU only).

* hand-derived closed forms of Eq. 5 / Eq. 7 / Eq. 12 (tests/golden),
* dense 2^n conjugation e^{-i tau P/2} H e^{i tau P/2} built from np.kron of
  the textbook Pauli matrices, dense <Omega|H|Omega>, exact diagonalisation,
* brute force over every Pauli string at tiny n (DIS rule of App. A),
* invariants that hold at any size (norm, identity term, inverse and group
  laws of the rotation, variational bound),
* sorting-based brute force for the compression step.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests import dense

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "worked_examples.json")


def _ev(expr, **kw):
    env = {"cos": math.cos, "sin": math.sin, "pi": math.pi}
    env.update(kw)
    return float(eval(expr, {"__builtins__": {}}, env))


def _from_words(n, terms):
    W = (n + 63) // 64
    xs, zs, cs = [], [], []
    for word, c in terms.items():
        x, z = dense.bits(word, W)
        xs.append(x)
        zs.append(z)
        cs.append(c)
    return np.array(xs, np.uint64).reshape(-1, W), np.array(zs, np.uint64).reshape(-1, W), np.array(cs, float)


def _words(o):
    x, z, c = o.export()
    return {dense.letters(o.n, x[i], z[i]): c[i] for i in range(len(c))}


def _random_angles(n, rng):
    return rng.uniform(0, np.pi, n), rng.uniform(0, 2 * np.pi, n)


# --------------------------------------------------------------------------- golden


@pytest.mark.parametrize("case", json.load(open(GOLDEN))["dress"])
@pytest.mark.parametrize("t", [0.0, 0.3, -1.7, 2.9])
def test_worked_dress(case, t):
    n = case["n"]
    o = oracle.Oracle(n, *_from_words(n, case["H"]))
    gx, gz = dense.bits(case["P"], o.W)
    o.dress(gx, gz, t)
    got = _words(o)
    want = {k: _ev(v, t=t) for k, v in case["expect"].items()}
    for k in set(got) | set(want):
        assert got.get(k, 0.0) == pytest.approx(want.get(k, 0.0), abs=1e-14), k


@pytest.mark.parametrize("th,ph", [(0.3, 1.1), (2.5, -0.4), (np.pi / 2, 3.0)])
def test_worked_energy_abc_gradient(th, ph):
    gold = json.load(open(GOLDEN))
    for case in gold["energy"]:
        o = oracle.Oracle(case["n"], *_from_words(case["n"], case["H"]))
        assert o.energy([th], [ph]) == pytest.approx(_ev(case["E"], th=th, ph=ph), abs=1e-14)
    for case in gold["abc"]:
        o = oracle.Oracle(case["n"], *_from_words(case["n"], case["H"]))
        gx, gz = dense.bits(case["P"], o.W)
        a, b, c = o.abc(gx, gz, [th], [ph])
        assert a == pytest.approx(_ev(case["A"], th=th, ph=ph), abs=1e-14)
        assert b == pytest.approx(_ev(case["B"], th=th, ph=ph), abs=1e-14)
        assert c == pytest.approx(_ev(case["C"], th=th, ph=ph), abs=1e-14)
    for case in gold["gradient"]:
        o = oracle.Oracle(case["n"], *_from_words(case["n"], case["H"]))
        gx, gz = dense.bits(case["P"], o.W)
        assert o.gradient(gx, gz, [th], [ph]) == pytest.approx(_ev(case["g"], th=th, ph=ph), abs=1e-14)
    for case in gold["minimum"]:
        o = oracle.Oracle(case["n"], *_from_words(case["n"], case["H"]))
        gx, gz = dense.bits(case["P"], o.W)
        a, b, c = o.abc(gx, gz, [th], [ph])
        tau = math.atan2(-c, -b)
        want = _ev(case["tau_star"], th=th, ph=ph)
        assert math.remainder(tau - want, 2 * math.pi) == pytest.approx(0.0, abs=1e-12)
        o.dress(gx, gz, tau)
        assert o.energy([th], [ph]) == pytest.approx(_ev(case["E_min"], th=th, ph=ph), abs=1e-14)


# --------------------------------------------------------------------------- dense


def test_letter_algebra_exhaustive_two_qubits():
    """Every (T, P) pair of 2-qubit strings, dressed, equals dense conjugation."""
    words = ["".join(p) for p in itertools.product("IXYZ", repeat=2)]
    for T in words:
        for P in words[1:]:
            for t in (0.37, -1.2):
                o = oracle.Oracle(2, *_from_words(2, {T: 1.0}))
                gx, gz = dense.bits(P, 1)
                Hd = dense.conjugate(dense.pauli_matrix(T), P, t)
                o.dress(gx, gz, t)
                got = _words(o)
                for W_ in words:
                    ref = dense.decompose_coefficient(Hd, W_)
                    assert abs(ref.imag) < 1e-12
                    assert got.get(W_, 0.0) == pytest.approx(ref.real, abs=1e-13), (T, P, t, W_)


@pytest.mark.parametrize("n,m,seed", [(3, 20, 1), (5, 60, 2), (8, 150, 3)])
def test_dress_matches_dense_conjugation(n, m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    n_, x, z, c = synth.random_hamiltonian(n, m, seed, scale="normal")
    Hm = dense.dense(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    for k in range(3):
        gx, gz = synth.random_generator(n, rng)
        t = float(rng.uniform(-np.pi, np.pi))
        o.dress(gx, gz, t)
        Hm = dense.conjugate(Hm, dense.letters(n, gx, gz), t)
    x2, z2, c2 = o.export()
    rec = dense.dense(n, x2, z2, c2)
    assert np.abs(rec - Hm).max() < 1e-12
    for i in range(len(c2)):                       # every stored coefficient is Tr(P_k H)/2^n
        ref = dense.decompose_coefficient(Hm, dense.letters(n, x2[i], z2[i]))
        assert c2[i] == pytest.approx(ref.real, abs=1e-12)


@pytest.mark.parametrize("n,seed", [(4, 5), (7, 6)])
def test_energy_abc_gradient_match_dense(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, 80, seed, scale="normal")
    Hm = dense.dense(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    th, ph = _random_angles(n, rng)
    psi = dense.qmf_state(th, ph)
    assert o.energy(th, ph) == pytest.approx(dense.expval(Hm, psi).real, abs=1e-12)
    for _ in range(4):
        gx, gz = synth.random_generator(n, rng)
        P = dense.letters(n, gx, gz)
        a, b, cc = o.abc(gx, gz, th, ph)
        for t in (0.0, 0.4, -2.2, 3.0):
            e = dense.expval(dense.conjugate(Hm, P, t), psi).real
            assert a + b * math.cos(t) + cc * math.sin(t) == pytest.approx(e, abs=1e-12)
        # Eq. 7 (paper sign) and a central difference of the dense energy
        g_paper = dense.expval(Hm @ dense.pauli_matrix(P), psi).imag
        h = 1e-5
        fd = (dense.expval(dense.conjugate(Hm, P, h), psi).real
              - dense.expval(dense.conjugate(Hm, P, -h), psi).real) / (2 * h)
        g = o.gradient(gx, gz, th, ph)
        assert g == pytest.approx(-g_paper, abs=1e-12)
        assert g == pytest.approx(fd, abs=1e-8)
        assert g == pytest.approx(cc, abs=1e-12)


@pytest.mark.parametrize("kind", ["basis", "uniform"])
def test_dis_rule_brute_force(kind):
    """Every Pauli string on 3 qubits: the ones with a non-zero gradient at a
    z-eigenstate are exactly those with odd Y parity and a flip set that some
    term of H has (App. A); the oracle's candidates carry the dense gradient."""
    n = 3
    rng = np.random.Generator(np.random.PCG64(11))
    _, x, z, c = synth.random_hamiltonian(n, 12, 11, density=0.5, scale="normal")
    Hm = dense.dense(n, x, z, c)
    if kind == "basis":
        th = np.array([np.pi, 0.0, np.pi])
        ph = np.zeros(n)
    else:
        th, ph = _random_angles(n, rng)
    psi = dense.qmf_state(th, ph)
    flips = {tuple(l in "XY" for l in dense.letters(n, x[i], z[i])) for i in range(len(c))}
    o = oracle.Oracle(n, x, z, c)
    cx, cz, cg = o.dis(th, ph)
    got = {dense.letters(n, cx[i], cz[i]): cg[i] for i in range(len(cg))}
    for word in ("".join(p) for p in itertools.product("IXYZ", repeat=n)):
        g = -dense.expval(Hm @ dense.pauli_matrix(word), psi).imag
        fl = tuple(l in "XY" for l in word)
        if kind == "basis" and abs(g) > 1e-12:
            assert word.count("Y") % 2 == 1 and fl in flips, word
        if word in got:
            assert got[word] == pytest.approx(g, abs=1e-12)
    # one representative per non-empty flip set of H, Y on the lowest flipped qubit
    reps = set()
    for fl in flips:
        if any(fl):
            lo = fl.index(True)
            reps.add("".join("Y" if j == lo else ("X" if fl[j] else "I") for j in range(n)))
    assert set(got) == reps
    # order: |g| descending (coarsened to 2^-32 relative), then key ascending
    mags = [abs(v) for v in cg]
    assert all(mags[i] >= mags[i + 1] * (1 - 2 ** -30) for i in range(len(mags) - 1))


def test_dis_ties_in_canonical_key_order():
    """Exact ties of |g| are ordered by the canonical key (x as an unsigned
    integer, then z), ascending.  H = 0.5 X0 + 0.5 X1 + 0.5 X0 X2 + 0.25 X2 +
    0.3 Z0 at the z-eigenstate theta = (pi, 0, pi): the representatives Y0,
    Y1 and Y0 X2 all have |g| = 0.5 exactly (from X Y = i Z and <Z> = -1, +1,
    -1), Y2 has 0.25; so the order is Y0 (x = 1), Y1 (x = 2), Y0 X2 (x = 5),
    then Y2.  A reversed tie order fails."""
    n = 3
    x, z, c = _from_words(n, {"XII": 0.5, "IXI": 0.5, "XIX": 0.5, "IIX": 0.25, "ZII": 0.3})
    th = np.array([np.pi, 0.0, np.pi])
    ph = np.zeros(n)
    o = oracle.Oracle(n, x, z, c)
    cx, cz, cg = o.dis(th, ph)
    order = [dense.letters(n, cx[i], cz[i]) for i in range(len(cg))]
    assert order == ["YII", "IYI", "YIX", "IIY"]
    psi = dense.qmf_state(th, ph)
    Hm = dense.dense(n, x, z, c)
    for word, g in zip(order, cg):
        assert g == pytest.approx(-dense.expval(Hm @ dense.pauli_matrix(word), psi).imag, abs=1e-14)
    assert [abs(v) for v in cg] == pytest.approx([0.5, 0.5, 0.5, 0.25], abs=1e-15)


# --------------------------------------------------------------------------- invariants


def _sq(o):
    return float(np.sum(o.export()[2] ** 2))


def test_rotation_invariants():
    n = 12
    rng = np.random.Generator(np.random.PCG64(21))
    _, x, z, c = synth.random_hamiltonian(n, 400, 21)
    x = np.vstack([x, np.zeros((1, 1), np.uint64)])
    z = np.vstack([z, np.zeros((1, 1), np.uint64)])
    c = np.append(c, 3.25)                            # identity term
    base = oracle.Oracle(n, x, z, c)
    ref = base.as_dict()
    for k in range(4):
        gx, gz = synth.random_generator(n, rng)
        t1, t2 = rng.uniform(-3, 3, 2)
        o = oracle.Oracle(n, x, z, c)
        o.dress(gx, gz, t1)
        d = o.as_dict()
        assert d[(0,) * 2] == 3.25                           # identity untouched
        assert _sq(o) == pytest.approx(_sq(base), rel=1e-13)  # rotation of pairs
        for key in d:                                        # real strings stay even-Y
            assert bin(key[0] & key[1]).count("1") % 2 == 0
        o.dress(gx, gz, -t1)                                 # inverse
        back = o.as_dict()
        for key in set(back) | set(ref):
            assert back.get(key, 0.0) == pytest.approx(ref.get(key, 0.0), abs=1e-13)
        o1 = oracle.Oracle(n, x, z, c)
        o1.dress(gx, gz, t1)
        o1.dress(gx, gz, t2)
        o2 = oracle.Oracle(n, x, z, c)
        o2.dress(gx, gz, t1 + t2)                            # one-parameter group
        a, b = o1.as_dict(), o2.as_dict()
        for key in set(a) | set(b):
            assert a.get(key, 0.0) == pytest.approx(b.get(key, 0.0), abs=1e-13)
        o3 = oracle.Oracle(n, x, z, c)
        o3.dress(gx, gz, math.pi)                           # pi negates anticommuting strings
        d3 = o3.as_dict()
        for key, v in ref.items():
            comm = (bin((key[0] & int(gz[0])) ^ (key[1] & int(gx[0]))).count("1") % 2) == 0
            assert d3[key] == pytest.approx(v if comm else -v, abs=1e-13)


def test_commuting_generator_is_identity():
    n = 6
    _, x, z, c = synth.random_hamiltonian(n, 100, 4)
    # a generator commuting with every term: Z on a qubit where no term has X or Y
    x[:, 0] &= ~np.uint64(1 << 5)
    o = oracle.Oracle(n, x, z, c)
    ref = o.as_dict()
    o.dress(np.array([0], np.uint64), np.array([1 << 5], np.uint64), 0.77)
    assert o.as_dict() == ref


def test_jw8_iterations_isospectral_variational_and_dense():
    """Three oracle iterations of the 8-qubit JW workload, checked against the
    dense product of the recorded rotations: energies, gradients, the top-2
    choice, monotone energy, the variational bound and the unchanged spectrum."""
    w = synth.WORKLOADS["jw8"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    H0 = dense.dense(n, x, z, c)
    lam = np.linalg.eigvalsh(H0)
    psi = dense.qmf_state(th, ph)
    o = oracle.Oracle(n, x, z, c)
    Hm = H0.copy()
    e_prev = dense.expval(H0, psi).real
    for it in range(w.n_iter):
        cx, cz, cg = o.dis(th, ph)
        for i in range(len(cg)):
            P = dense.letters(n, cx[i], cz[i])
            assert cg[i] == pytest.approx(-dense.expval(Hm @ dense.pauli_matrix(P), psi).imag, abs=1e-11)
        rec = o.iterate(th, ph, w.n_gen, w.eps, w.max_terms)
        assert len(rec["tau"]) == w.n_gen
        for k in range(w.n_gen):
            assert dense.letters(n, rec["gx"][k], rec["gz"][k]) == dense.letters(n, cx[k], cz[k])
            P = dense.letters(n, rec["gx"][k], rec["gz"][k])
            Hm = dense.conjugate(Hm, P, rec["tau"][k])
            e = dense.expval(Hm, psi).real
            assert e <= e_prev + 1e-12                       # tau = 0 was admissible
            e_prev = e
        assert rec["energy"] == pytest.approx(e_prev, abs=1e-11)
        assert rec["energy"] >= lam[0] - 1e-10
        x2, z2, c2 = o.export()
        assert np.abs(dense.dense(n, x2, z2, c2) - Hm).max() < 1e-11
    assert np.allclose(np.linalg.eigvalsh(Hm), lam, atol=1e-10)


# --------------------------------------------------------------------------- compression and load


def test_prune_matches_sorting_brute_force():
    n = 10
    rng = np.random.Generator(np.random.PCG64(3))
    _, x, z, c = synth.random_hamiltonian(n, 500, 3)
    c = np.round(c, 2)                                 # many exact ties in |c|
    c[c == 0] = 0.01
    c = c * rng.choice([-1.0, 1.0], len(c))
    for eps, cap in [(0.0, 0), (0.05, 0), (0.0, 123), (0.05, 77), (0.3, 10_000)]:
        o = oracle.Oracle(n, x, z, c)
        removed = o.prune(eps, cap)
        rows = [(tuple(x[i][::-1]), tuple(z[i][::-1]), c[i]) for i in range(len(c))]
        rows = [r for r in rows if abs(r[2]) >= eps]
        rows.sort(key=lambda r: (-abs(r[2]), r[0], r[1]))
        if cap > 0:
            rows = rows[:cap]
        want = {(r[0][::-1], r[1][::-1]): r[2] for r in rows}
        gx, gz, gc = o.export()
        got = {(tuple(gx[i]), tuple(gz[i])): gc[i] for i in range(len(gc))}
        assert got == {k: v for k, v in want.items()}
        assert removed == len(c) - len(want)


def test_load_sums_duplicates_and_drops_zeros():
    x = np.array([[1], [1], [2], [2], [3]], np.uint64)
    z = np.array([[0], [0], [2], [2], [0]], np.uint64)
    c = np.array([0.5, 0.25, 1.0, -1.0, 0.0])
    o = oracle.Oracle(3, x, z, c)
    assert o.as_dict() == {(1, 0): 0.75}
    assert len(oracle.Oracle(3)) == 0


def test_canonical_export_order():
    n = 70
    _, x, z, c = synth.random_hamiltonian(n, 300, 9)
    xs, zs, cs = oracle.Oracle(n, x, z, c).export()
    keys = [tuple(xs[i][::-1]) + tuple(zs[i][::-1]) for i in range(len(cs))]
    assert keys == sorted(keys)


def test_iteration_applies_the_term_limit_after_every_dress():
    """orc_iterate = the pinned primitives in App. A order: each dress followed by
    a cut to max_terms when exceeded, then (eps, max_terms) compression."""
    w = synth.WORKLOADS["jw8"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    cap = 500
    a = oracle.Oracle(n, x, z, c)
    ra = a.iterate(th, ph, 3, 1e-3, cap)
    b = oracle.Oracle(n, x, z, c)
    removed = 0
    for k in range(len(ra["tau"])):
        _, bb, cc = b.abc(ra["gx"][k], ra["gz"][k], th, ph)
        assert math.atan2(-cc, -bb) == ra["tau"][k]
        b.dress(ra["gx"][k], ra["gz"][k], ra["tau"][k])
        if len(b) > cap:
            removed += b.prune(0.0, cap)
    removed += b.prune(1e-3, cap)
    assert a.as_dict() == b.as_dict()
    assert ra["removed"] == removed and removed > 0
    assert ra["energy"] == b.energy(th, ph)


# ---------------------------------------------------------------------------
# Angle and amplitude derivatives of the dressed QMF energy (Eq. 3, Eq. 5, Eq. 12)


def _dense_dressed_energy(n, x, z, c, word, tau, theta, phi):
    Hm = dense.dense(n, x, z, c)
    if word is not None:
        Hm = dense.conjugate(Hm, word, tau)
    return float(dense.expval(Hm, dense.qmf_state(theta, phi)).real)


@pytest.mark.parametrize("n,with_gen", [(3, False), (3, True), (4, True), (5, False)])
def test_energy_gradients_match_dense_finite_differences(n, with_gen):
    """Every derivative against a central difference of the dense energy
    <Omega| U H U^dagger |Omega> (np.kron statevectors, dense conjugation)."""
    rng = np.random.Generator(np.random.PCG64(40 + n + 7 * with_gen))
    _, x, z, c = synth.random_hamiltonian(n, 12, 90 + n)
    theta = rng.uniform(0, np.pi, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    o = oracle.Oracle(n, x, z, c)
    word, gx, gz, tau = None, None, None, 0.0
    if with_gen:
        gx, gz = synth.random_generator(n, rng, weight=2)
        word = dense.letters(n, np.asarray(gx).reshape(-1), np.asarray(gz).reshape(-1))
        tau = float(rng.uniform(-1.5, 1.5))
    e, dt, dp, dtau = o.energy_gradients(theta, phi, gx, gz, tau)
    assert e == pytest.approx(_dense_dressed_energy(n, x, z, c, word, tau, theta, phi), abs=1e-12)
    h = 1e-6
    for k in range(n):
        for arr, got in ((theta, dt[k]), (phi, dp[k])):
            up, dn = arr.copy(), arr.copy()
            up[k] += h
            dn[k] -= h
            args_up = (theta, up) if arr is phi else (up, phi)
            args_dn = (theta, dn) if arr is phi else (dn, phi)
            fd = (_dense_dressed_energy(n, x, z, c, word, tau, args_up[0], args_up[1])
                  - _dense_dressed_energy(n, x, z, c, word, tau, args_dn[0], args_dn[1])) / (2 * h)
            assert got == pytest.approx(fd, abs=2e-8), (k, got, fd)
    if with_gen:
        fd = (_dense_dressed_energy(n, x, z, c, word, tau + h, theta, phi)
              - _dense_dressed_energy(n, x, z, c, word, tau - h, theta, phi)) / (2 * h)
        assert dtau == pytest.approx(fd, abs=2e-8)
    else:
        assert dtau == 0.0


@pytest.mark.parametrize("word,theta,phi", [("X", [0.7], [0.3]), ("Y", [1.9], [2.2]), ("Z", [0.4], [1.0]),
                                            ("XZ", [0.8, 2.1], [0.5, 1.3])])
def test_energy_gradients_closed_forms(word, theta, phi):
    """<X> = sin t cos p, <Y> = sin t sin p, <Z> = cos t per qubit, differentiated by hand."""
    n = len(word)
    x, z, c = _from_words(n, {word: 1.5})
    e, dt, dp, _ = oracle.Oracle(n, x, z, c).energy_gradients(theta, phi)
    t, p = np.array(theta), np.array(phi)
    f = {"X": (np.sin(t) * np.cos(p), np.cos(t) * np.cos(p), -np.sin(t) * np.sin(p)),
         "Y": (np.sin(t) * np.sin(p), np.cos(t) * np.sin(p), np.sin(t) * np.cos(p)),
         "Z": (np.cos(t), -np.sin(t), np.zeros_like(t))}
    val = np.array([f[l][0][j] for j, l in enumerate(word)])
    for k, l in enumerate(word):
        others = np.prod(np.delete(val, k))
        assert dt[k] == pytest.approx(1.5 * f[l][1][k] * others, abs=1e-14)
        assert dp[k] == pytest.approx(1.5 * f[l][2][k] * others, abs=1e-14)
    assert e == pytest.approx(1.5 * np.prod(val), abs=1e-14)


@pytest.mark.parametrize("n", [6, 9])
def test_energy_gradient_in_tau_at_zero_is_eq7(n):
    """dE/dtau at tau = 0 equals the Eq. 7 gradient (orc_gradient, pinned on its own)."""
    rng = np.random.Generator(np.random.PCG64(300 + n))
    _, x, z, c = synth.random_hamiltonian(n, 60, 500 + n)
    theta = rng.uniform(0, np.pi, n)
    phi = rng.uniform(0, 2 * np.pi, n)
    o = oracle.Oracle(n, x, z, c)
    for _ in range(3):
        gx, gz = synth.random_generator(n, rng, weight=3)
        _, _, _, dtau = o.energy_gradients(theta, phi, gx, gz, 0.0)
        assert dtau == pytest.approx(o.gradient(gx, gz, theta, phi), abs=1e-12)


def test_phi_gradients_vanish_at_basis_states():
    """On a z-eigenstate every single-qubit state is |0> or |1>, where phi is a
    global phase of the qubit: dE/dphi = 0 (sin(pi) ~ 1e-16 aside)."""
    n = 7
    _, x, z, c = synth.random_hamiltonian(n, 80, 77)
    theta = np.where(np.arange(n) < 3, np.pi, 0.0)
    phi = np.linspace(0.1, 2.0, n)
    _, dt, dp, _ = oracle.Oracle(n, x, z, c).energy_gradients(theta, phi)
    assert np.max(np.abs(dp)) < 1e-14 * max(1.0, np.abs(c).sum())
