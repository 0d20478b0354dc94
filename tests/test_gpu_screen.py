"""Learned term screening: features, future energies (the training target),
the tensor-core perceptron and the learned term limit."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)


def _popc_rows(x):
    return np.array([sum(bin(int(w)).count("1") for w in row) for row in np.atleast_2d(x)])


def _single_energy(n, x, z, th, ph, gens=(), taus=()):
    o = oracle.Oracle(n, x.reshape(1, -1), z.reshape(1, -1), np.array([1.0]))
    for (gx, gz), t in zip(gens, taus):
        o.dress(gx, gz, t)
    return o.energy(th, ph)


@pytest.mark.parametrize("n,angles", [(8, "uniform"), (24, "basis"), (70, "uniform")])
def test_future_energies_match_dressed_single_strings(n, angles):
    """E_fut(T) against the oracle dressing {T: 1} generator by generator."""
    rng = np.random.Generator(np.random.PCG64(n))
    _, x, z, c = synth.random_hamiltonian(n, 120, 60 + n, density=min(0.5, 10 / n))
    th, ph = synth.qmf_angles(n, angles, seed=n)
    gens = [synth.random_generator(n, rng, weight=2) for _ in range(3)]
    taus = rng.uniform(-1.5, 1.5, 3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    ex, ez, ec = iqcc.iqcc_export(H)
    fut = iqcc.iqcc_future_energies(H, th, ph, np.array([g[0] for g in gens]), np.array([g[1] for g in gens]), taus)
    for i in range(len(ec)):
        ref = _single_energy(n, ex[i], ez[i], th, ph, gens, taus)
        assert fut[i] == pytest.approx(ref, abs=1e-12), i


@pytest.mark.parametrize("n,density", [(12, 0.2), (100, 0.2), (200, 0.5)])
def test_features_match_their_definition(n, density):
    """Including strings past the saturation of the flip and Y counts (200 qubits, half of them set)."""
    rng = np.random.Generator(np.random.PCG64(5 + n))
    _, x, z, c = synth.random_hamiltonian(n, 300, 80 + n, density=density)
    th, ph = synth.qmf_angles(n, "uniform", seed=2)
    gens = [synth.random_generator(n, rng, weight=3) for _ in range(2)]
    gx = np.array([g[0] for g in gens])
    gz = np.array([g[1] for g in gens])
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    ex, ez, ec = iqcc.iqcc_export(H)
    f = iqcc.iqcc_term_features(H, th, ph, gx, gz)
    G = np.bitwise_or.reduce(np.concatenate([gx, gz]), axis=0)
    for i in range(len(ec)):
        xi, zi = ex[i], ez[i]
        flips = _popc_rows(xi)[0]
        fov = _popc_rows(xi & G)[0]
        want = [math.log10(abs(ec[i])) / 8, min(flips, 16) / 16, min(_popc_rows(xi & zi)[0], 16) / 16,
                _popc_rows(zi & ~xi & G)[0] / 8, _popc_rows((xi | zi) & G)[0] / 8, fov / 8,
                _single_energy(n, xi, zi, th, ph), 1.0 if (flips > 0 and fov == flips) else 0.0]
        assert np.allclose(f[i], want, rtol=1e-5, atol=1e-6), (i, f[i], want)  # FP32 features


def _random_model(seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    w1 = rng.standard_normal((256, 8)).astype(np.float32) * 0.5
    b1 = rng.standard_normal(256).astype(np.float32) * 0.1
    w2 = rng.standard_normal((256, 256)).astype(np.float32) / 16
    b2 = rng.standard_normal(256).astype(np.float32) * 0.1
    w3 = rng.standard_normal(256).astype(np.float32) / 16
    return w1, b1, w2, b2, w3, np.float32(-1.0)


def _bf16(a):
    """Round float32 to bfloat16 (nearest even) and back."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def _reference_scores(feat, model):
    """Plain FP32 forward pass with the kernel's BF16 roundings (inputs, weights, hidden layer 1)."""
    w1, b1, w2, b2, w3, b3 = model
    h1 = np.maximum(_bf16(feat) @ _bf16(w1).T + b1, 0)
    h2 = np.maximum(_bf16(h1) @ _bf16(w2).T + b2, 0)
    return h2 @ w3 + b3


@pytest.mark.parametrize("n,m", [(20, 1000), (100, 5003)])
def test_perceptron_scores_match_a_plain_forward_pass(n, m):
    rng = np.random.Generator(np.random.PCG64(n))
    _, x, z, c = synth.random_hamiltonian(n, m, 90 + n, density=0.2)
    th, ph = synth.qmf_angles(n, "uniform", seed=4)
    gens = [synth.random_generator(n, rng, weight=3) for _ in range(2)]
    gx = np.array([g[0] for g in gens])
    gz = np.array([g[1] for g in gens])
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    model = _random_model(n)
    iqcc.iqcc_set_screening_model(H, *model)
    s = iqcc.iqcc_term_scores(H, th, ph, gx, gz)
    ref = _reference_scores(iqcc.iqcc_term_features(H, th, ph, gx, gz), model)
    assert np.allclose(s, ref, rtol=2e-3, atol=2e-3 * np.abs(ref).max()), np.abs(s - ref).max()


def test_learned_term_limit_keeps_the_best_scores():
    n = 30
    rng = np.random.Generator(np.random.PCG64(3))
    _, x, z, c = synth.random_hamiltonian(n, 20_000, 33, density=0.3)
    th, ph = synth.qmf_angles(n, "basis")
    gx, gz = synth.random_generator(n, rng, weight=3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_set_screening_model(H, *_random_model(7))
    iqcc.iqcc_set_screening_floor(H, 0.0)
    s = iqcc.iqcc_term_scores(H, th, ph, gx, gz)
    ex, ez, ec = iqcc.iqcc_export(H)
    keep = 7000
    rank = np.maximum(s, -1000).astype(np.float64) + 1024.0   # the library's key: exact and increasing
    order = sorted(range(len(s)), key=lambda i: (-rank[i], i))  # export order is canonical: index = key order
    expect = {(ex[i].tobytes(), ez[i].tobytes()) for i in order[:keep]}
    removed = iqcc.iqcc_prune_learned(H, 0.0, keep, th, ph, gx, gz)
    assert removed == len(s) - keep and len(H) == keep
    kx, kz, kc = iqcc.iqcc_export(H)
    assert {(a.tobytes(), b.tobytes()) for a, b in zip(kx, kz)} == expect


@pytest.mark.parametrize("m,floor", [(20_000, 0.4), (20_000, 1.0), (150_000, 0.5)])
def test_learned_term_limit_keeps_its_magnitude_floor(m, floor):
    """The floor x limit largest |C| are kept first, then the best scores among
    the other terms (150,000 terms: the floor's threshold comes out of the
    12-bit radix select, then an exact pick inside its bucket)."""
    n = 30
    rng = np.random.Generator(np.random.PCG64(4))
    _, x, z, c = synth.random_hamiltonian(n, m, 35, density=0.3)
    th, ph = synth.qmf_angles(n, "basis")
    gx, gz = synth.random_generator(n, rng, weight=3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_set_screening_model(H, *_random_model(8))
    iqcc.iqcc_set_screening_floor(H, floor)
    s = iqcc.iqcc_term_scores(H, th, ph, gx, gz)
    ex, ez, ec = iqcc.iqcc_export(H)
    keep = int(0.35 * len(ec))
    n_mag = int(floor * keep)
    by_mag = sorted(range(len(ec)), key=lambda i: (-abs(ec[i]), i))
    top = set(by_mag[:n_mag])
    rank = np.maximum(s, -1000).astype(np.float64) + 1024.0
    rest = sorted((i for i in range(len(ec)) if i not in top), key=lambda i: (-rank[i], i))
    chosen = list(top) + rest[:keep - len(top)]
    expect = {(ex[i].tobytes(), ez[i].tobytes()) for i in chosen}
    removed = iqcc.iqcc_prune_learned(H, 0.0, keep, th, ph, gx, gz)
    assert removed == len(ec) - keep and len(H) == keep
    kx, kz, kc = iqcc.iqcc_export(H)
    assert {(a.tobytes(), b.tobytes()) for a, b in zip(kx, kz)} == expect


def test_magnitude_floor_with_more_equal_magnitudes_than_a_bucket_holds():
    """150,000 terms of |C| = 1: the floor's threshold bucket cannot be narrowed
    below 65,536 rows; every term ties at the threshold, so the limit keeps the
    first terms in canonical order."""
    n = 30
    rng = np.random.Generator(np.random.PCG64(6))
    _, x, z, c = synth.random_hamiltonian(n, 150_000, 36, density=0.3)
    c = np.where(rng.integers(0, 2, len(c)) == 1, 1.0, -1.0)
    th, ph = synth.qmf_angles(n, "basis")
    gx, gz = synth.random_generator(n, rng, weight=3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_set_screening_model(H, *_random_model(9))
    ex, ez, ec = iqcc.iqcc_export(H)
    keep = 40_000
    removed = iqcc.iqcc_prune_learned(H, 0.0, keep, th, ph, gx, gz)
    assert removed == len(ec) - keep and len(H) == keep
    kx, kz, kc = iqcc.iqcc_export(H)
    assert np.array_equal(kx, ex[:keep]) and np.array_equal(kz, ez[:keep]) and np.array_equal(kc, ec[:keep])


def test_screening_floor_rejects_values_outside_the_unit_interval():
    _, x, z, c = synth.random_hamiltonian(10, 100, 3)
    H = iqcc.iqcc_load_hamiltonian(10, x, z, c)
    for bad in (-0.1, 1.5, float("nan")):
        with pytest.raises(iqcc.IqccError):
            iqcc.iqcc_set_screening_floor(H, bad)
    iqcc.iqcc_set_screening_floor(H, 0.0)
    iqcc.iqcc_set_screening_floor(H, 1.0)


def test_iteration_with_learned_screening_runs_and_respects_the_cap():
    w = synth.WORKLOADS["jw24"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    with pytest.raises(iqcc.IqccError):   # no model yet
        iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 20_000, screening=1)
    iqcc.iqcc_set_screening_model(H, *_random_model(11))
    for _ in range(3):
        r = iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 20_000, screening=1)
        assert r["M"] <= 20_000 and np.isfinite(r["energy"])


def test_shipped_model_screens_within_the_target_on_a_held_out_problem():
    """The trained model (screening/model_jw.npz, from screening/train.py) on a
    22-qubit problem outside its training set: after 4 iterations with a term
    limit of 30% of the untruncated run's size, the energy stays within 1e-5 Ha
    of the untruncated one (the magnitude limit's error is reported beside it)."""
    from paper_2603_08883_gb300.screening import load_model, train
    n, x, z, c, th, ph = train.problem(11, 4200)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    for _ in range(4):
        r = iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 0)
    e_ref, cap = r["energy"], int(0.3 * r["M"])
    errs = {}
    for mode in (0, 1):
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
        iqcc.iqcc_set_screening_model(H, *load_model())
        for _ in range(4):
            r = iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, cap, screening=mode)
        assert r["M"] <= cap
        errs[mode] = abs(r["energy"] - e_ref)
    assert errs[1] < 1e-5, errs
    assert errs[1] <= errs[0], errs
