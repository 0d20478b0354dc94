"""GPU parity: every entry point of the C ABI against the CPU oracle on the
same seeded inputs (sizes the oracle finishes in seconds, several tiles and a
ragged tail; word counts 1, 2, 3 and 4; the degenerate cases)."""
import math

import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth
from tests.compare import ABS, REL, compare

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)

SIZES = [(1, 3, 1), (7, 3000, 2), (24, 40_037, 3), (64, 20_011, 4), (65, 30_029, 5), (100, 50_021, 6),
         (130, 20_003, 7), (200, 12_007, 8)]


def _with_dups(n, m, seed):
    """Random H plus repeated keys and an exact cancellation, shuffled."""
    n_, x, z, c = synth.random_hamiltonian(n, m, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 99))
    k = max(1, len(c) // 10)
    pick = rng.integers(0, len(c), k)
    x = np.vstack([x, x[pick]])
    z = np.vstack([z, z[pick]])
    c = np.concatenate([c, rng.standard_normal(k)])
    if len(c) > 2:                      # one key cancels exactly to zero
        x = np.vstack([x, x[:1]])
        z = np.vstack([z, z[:1]])
        c = np.append(c, -np.sum(c[np.all(x[:-1] == x[0], 1) & np.all(z[:-1] == z[0], 1)]))
    perm = rng.permutation(len(c))
    return x[perm], z[perm], c[perm]


@pytest.mark.parametrize("n,m,seed", SIZES)
def test_load_and_export_canonical(n, m, seed):
    x, z, c = _with_dups(n, m, seed)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    gx, gz, gc = iqcc.iqcc_export(H)
    ox, oz, oc = o.export()
    assert len(gc) == len(oc) == len(H)
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz)      # same keys, same canonical order
    assert np.array_equal(gc, oc)                                   # sums in input order: bit-exact


@pytest.mark.parametrize("n,m,seed", SIZES)
def test_dress_matches_oracle(n, m, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, m, seed)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    gens = [synth.random_generator(n, rng) for _ in range(4)]
    taus = rng.uniform(-math.pi, math.pi, 4)
    for (gx, gz), t in zip(gens, taus):
        o.dress(gx, gz, t)
    assert iqcc.iqcc_dress(H, np.array([g[0] for g in gens]), np.array([g[1] for g in gens]), taus) == 4
    bad = compare(iqcc.iqcc_export(H), o.export())
    assert not bad, bad[:5]
    assert len(H) == len(o)                      # eps = 0: no key is dropped on either side


def test_dress_pairs_present_and_absent():
    """A generator whose partners are all present (pure rotations) and one whose
    partners are all absent (pure appends), with the exact key count."""
    n = 10
    _, x, z, c = synth.random_hamiltonian(n, 500, 17)
    P = (np.array([0b11], np.uint64), np.array([0b01], np.uint64))   # Y0 X1
    x2 = np.vstack([x, x ^ P[0]])
    z2 = np.vstack([z, z ^ P[1]])
    c2 = np.concatenate([c, c[::-1]])
    o = oracle.Oracle(n, x2, z2, c2)
    H = iqcc.iqcc_load_hamiltonian(n, x2, z2, c2)
    m0 = len(H)
    iqcc.iqcc_dress(H, P[0], P[1], [0.7])
    o.dress(P[0], P[1], 0.7)
    assert len(H) == m0                          # every partner present: no append
    assert not compare(iqcc.iqcc_export(H), o.export())


@pytest.mark.parametrize("n,seed", [(8, 1), (64, 2), (100, 3), (130, 4)])
@pytest.mark.parametrize("angles", ["basis", "uniform"])
def test_energy_and_abc_match_oracle(n, seed, angles):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, 30_000 if angles == "basis" else 5_000, seed, density=0.3)
    # plenty of diagonal and generator-matching strings
    x[: len(x) // 3] = 0
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, angles, seed)
    if angles == "basis":
        th = np.where(rng.random(n) < 0.5, np.pi, 0.0)
    e = iqcc.iqcc_qmf_energy(H, th, ph)
    assert e == pytest.approx(o.energy(th, ph), abs=1e-9)
    for k in range(3):
        gx, gz = synth.random_generator(n, rng)
        if k == 0 and len(x) > 10:                # a generator with the flip set of existing terms
            gx = x[len(x) // 2].copy()
            if not gx.any():
                gx[0] = np.uint64(3)
            gz = np.zeros_like(gx)
            low = int(np.nonzero(gx)[0][0])
            gz[low] = gx[low] & (~gx[low] + np.uint64(1))
        a = iqcc.iqcc_generator_abc(H, gx, gz, th, ph)
        b = o.abc(gx, gz, th, ph)
        assert np.allclose(a, b, rtol=0, atol=1e-9), (a, b)


@pytest.mark.parametrize("n,seed", [(6, 1), (24, 2), (100, 3)])
def test_dis_basis_matches_oracle(n, seed):
    _, x, z, c = synth.random_hamiltonian(n, 20_000, seed, density=0.15)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "basis")
    ox, oz, og = o.dis(th, ph)
    gx, gz, gg = iqcc.iqcc_dis_gradients(H, th, ph)
    assert len(gg) == len(og)
    ref = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(ox, oz, og)}
    got = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(gx, gz, gg)}
    assert ref.keys() == got.keys()
    for k in ref:
        assert got[k] == pytest.approx(ref[k], abs=1e-12 + 1e-12 * abs(ref[k]))
    # ordering: identical wherever the oracle's coarse |g| values are distinct
    top = min(len(og), 50)
    mag = np.abs(og)

    def separated(i, j):
        return j < 0 or j >= len(mag) or abs(mag[i] - mag[j]) > 1e-9 * mag[i]

    for i in range(top):
        if separated(i, i - 1) and separated(i, i + 1):
            assert (gx[i].tobytes(), gz[i].tobytes()) == (ox[i].tobytes(), oz[i].tobytes())
    # the capped query returns the head of the same order
    hx, hz, hg = iqcc.iqcc_dis_gradients(H, th, ph, cap=5)
    assert np.array_equal(hx, gx[:5])
    assert np.allclose(hg, gg[:5], rtol=1e-12, atol=1e-14)   # FP64 atomics: order of the group sums varies


@pytest.mark.parametrize("n,seed", [(5, 1), (12, 2), (70, 3)])
def test_dis_general_angles_and_given_candidates(n, seed):
    _, x, z, c = synth.random_hamiltonian(n, 300, seed, density=0.3)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "uniform", seed)
    ox, oz, og = o.dis(th, ph)
    gx, gz, gg = iqcc.iqcc_dis_gradients(H, th, ph)
    ref = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(ox, oz, og)}
    got = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(gx, gz, gg)}
    assert ref.keys() == got.keys()
    for k in ref:
        assert got[k] == pytest.approx(ref[k], abs=1e-10)
    rng = np.random.Generator(np.random.PCG64(seed))
    cand = [synth.random_generator(n, rng) for _ in range(37)]
    cx = np.array([a for a, b in cand])
    cz = np.array([b for a, b in cand])
    g = iqcc.iqcc_dis_gradients(H, th, ph, cx=cx, cz=cz)
    for i in range(len(cand)):
        assert g[i] == pytest.approx(o.gradient(cx[i], cz[i], th, ph), abs=1e-10)


def _dis_reps(x, rows):
    """DIS representatives (App. A): x = the flip set of a row, z = its lowest flipped qubit (one Y)."""
    cx = x[rows].copy()
    cz = np.zeros_like(cx)
    for i in range(len(rows)):
        for w in range(cx.shape[1]):
            v = int(cx[i, w])
            if v:
                cz[i, w] = np.uint64(v & -v)
                break
    return cx, cz


@pytest.mark.parametrize("n,seed", [(64, 21), (100, 22)])
def test_dis_general_angles_given_candidates_at_scale(n, seed):
    """General QMF angles, 1.2 x 10^5 strings and 80 given candidates (64 DIS
    representatives of flip sets present in H and 16 random generators): the
    M x K tiled gradient kernel over several candidate tiles.  Tolerance from
    the arithmetic: each g is a sum of M products of n factors, so its FP64
    error is bounded by about (n + log2 M) u sum_T |C_T|; the test allows
    1e-12 (|g| + sum_T |C_T|)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, 120_000, seed, density=0.12)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "uniform", seed)
    rows = rng.choice(np.nonzero(np.any(x != 0, axis=1))[0], 64, replace=False)
    cx, cz = _dis_reps(x, rows)
    extra = [synth.random_generator(n, rng) for _ in range(16)]
    cx = np.vstack([cx, [a for a, b in extra]])
    cz = np.vstack([cz, [b for a, b in extra]])
    g = iqcc.iqcc_dis_gradients(H, th, ph, cx=cx, cz=cz)
    l1 = float(np.sum(np.abs(c)))
    for i in range(len(cx)):
        ref = o.gradient(cx[i], cz[i], th, ph)
        assert abs(g[i] - ref) <= 1e-12 * (abs(ref) + l1), (i, g[i], ref)


def test_dis_general_angles_enumeration_at_moderate_size():
    """The enumerating general-angle path (every distinct flip set a
    candidate, each gradient summed over all of H) on 4,000 strings, against
    the oracle's candidate list, gradients (same bound as above) and order."""
    n = 40
    _, x, z, c = synth.random_hamiltonian(n, 4_000, 23, density=0.1)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "uniform", 23)
    ox, oz, og = o.dis(th, ph)
    gx, gz, gg = iqcc.iqcc_dis_gradients(H, th, ph)
    l1 = float(np.sum(np.abs(c)))
    ref = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(ox, oz, og)}
    got = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(gx, gz, gg)}
    assert ref.keys() == got.keys()
    for k in ref:
        assert abs(got[k] - ref[k]) <= 1e-12 * (abs(ref[k]) + l1)
    mag = np.abs(og)
    for i in range(min(len(og), 40)):
        lo = i == 0 or mag[i - 1] > mag[i] * (1 + 1e-9)
        hi = i + 1 >= len(og) or mag[i] > mag[i + 1] * (1 + 1e-9)
        if lo and hi:
            assert (gx[i].tobytes(), gz[i].tobytes()) == (ox[i].tobytes(), oz[i].tobytes())


@pytest.mark.parametrize("eps,cap", [(0.0, 0), (1e-3, 0), (0.0, 777), (1e-4, 5000), (0.0, 1), (10.0, 0)])
def test_prune_matches_oracle(eps, cap):
    n = 100
    _, x, z, c = synth.random_hamiltonian(n, 60_013, 31)
    rng = np.random.Generator(np.random.PCG64(5))
    c[: len(c) // 4] = np.round(c[: len(c) // 4], 3)            # exact |c| ties, some zeros
    c[len(c) // 4: len(c) // 2] = -c[: len(c) // 4][: len(c) // 2 - len(c) // 4]
    c = c * rng.choice([-1.0, 1.0], len(c))
    c[c == 0] = 1e-3
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    removed = iqcc.iqcc_prune(H, eps, cap)
    r_o = o.prune(eps, cap)
    assert removed == r_o
    gx, gz, gc = iqcc.iqcc_export(H)
    ox, oz, oc = o.export()
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gc, oc)


def test_empty_and_degenerate_cases():
    n = 9
    e = np.zeros((0, 1), np.uint64)
    H = iqcc.iqcc_load_hamiltonian(n, e, e, np.zeros(0))
    assert len(H) == 0
    assert iqcc.iqcc_dress(H, [3], [1], [0.5]) == 1
    assert iqcc.iqcc_prune(H, 1e-3, 5) == 0
    assert iqcc.iqcc_qmf_energy(H, np.zeros(n), np.zeros(n)) == 0.0
    x, z, c = iqcc.iqcc_export(H)
    assert len(c) == 0
    assert len(iqcc.iqcc_dis_gradients(H, np.zeros(n), np.zeros(n))[2]) == 0
    # all-zero input collapses to an empty Hamiltonian
    H = iqcc.iqcc_load_hamiltonian(n, np.ones((3, 1), np.uint64), np.zeros((3, 1), np.uint64), np.zeros(3))
    assert len(H) == 0
    # identity only; a generator commutes with it; tau = 0 and tau = 2 pi
    H = iqcc.iqcc_load_hamiltonian(n, np.zeros((1, 1), np.uint64), np.zeros((1, 1), np.uint64), np.array([2.5]))
    iqcc.iqcc_dress(H, [5], [4], [1.3])
    assert len(H) == 1 and iqcc.iqcc_export(H)[2][0] == 2.5
    _, x, z, c = synth.random_hamiltonian(n, 200, 3)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_dress(H, [1], [1], [0.0])
    o.dress([1], [1], 0.0)
    assert not compare(iqcc.iqcc_export(H), o.export())
    iqcc.iqcc_dress(H, [1], [1], [2 * math.pi])
    o.dress([1], [1], 2 * math.pi)
    assert not compare(iqcc.iqcc_export(H), o.export())


def test_capacity_error_leaves_h_unchanged():
    n = 20
    _, x, z, c = synth.random_hamiltonian(n, 3000, 8)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=len(c) + 10)
    before = iqcc.iqcc_export(H)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_dress(H, [0b111], [0b001], [0.3])   # anticommutes with about half, partners absent
    assert e.value.status == 4
    after = iqcc.iqcc_export(H)
    for a, b in zip(before, after):
        assert np.array_equal(a, b)
    iqcc.iqcc_prune(H, 1.0)                           # still usable


def test_arguments_rejected():
    n = 5
    _, x, z, c = synth.random_hamiltonian(n, 50, 1)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_dress(H, [1 << 7], [0], [0.1])
    assert e.value.status == 1
    with pytest.raises(iqcc.IqccError):
        iqcc.iqcc_dress(H, [1], [0], [float("nan")])
    assert len(H) == len(oracle.Oracle(n, x, z, c))


# ------------------------------------------------------------------ whole iterations


def test_jw8_iterations_free_running():
    """Configuration of the 8-qubit workload: 3 iterations x 2 generators with
    random QMF angles and no compression; the GPU screens, optimises and dresses
    on its own and must reproduce the oracle's choices and energies."""
    w = synth.WORKLOADS["jw8"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    for it in range(w.n_iter):
        ro = o.iterate(th, ph, w.n_gen, w.eps, w.max_terms)
        rg = iqcc.iqcc_iterate(H, th, ph, w.n_gen, w.eps, w.max_terms)
        assert np.array_equal(rg["gx"], ro["gx"]) and np.array_equal(rg["gz"], ro["gz"])
        assert np.allclose(rg["g"], ro["g"], rtol=1e-12, atol=1e-12)
        assert np.allclose(rg["tau"], ro["tau"], rtol=0, atol=1e-12)
        assert rg["energy"] == pytest.approx(ro["energy"], abs=1e-9)
        assert not compare(iqcc.iqcc_export(H), o.export())


def test_jw24_iterations_teacher_forced_and_free():
    """24-qubit workload: the GPU is given the oracle's generators and
    amplitudes (teacher forcing) and must reproduce the dressed Hamiltonian after
    every iteration; the free-running GPU energies of the same iterations must
    match too."""
    w = synth.WORKLOADS["jw24"]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    o = oracle.Oracle(n, x, z, c)
    Hf = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    Hs = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    for it in range(3):
        ro = o.iterate(th, ph, w.n_gen, w.eps, w.max_terms)
        rf = iqcc.iqcc_iterate(Hf, th, ph, w.n_gen, w.eps, w.max_terms, forced_x=ro["gx"], forced_z=ro["gz"],
                               forced_tau=ro["tau"])
        gpu, ref = iqcc.iqcc_export(Hf), o.export()
        bad = compare(gpu, ref, eps=w.eps)      # keys may differ only within 1e-12 relative of eps
        assert not bad, bad[:5]
        if np.array_equal(gpu[0], ref[0]) and np.array_equal(gpu[1], ref[1]):
            assert rf["removed"] == ro["removed"]
        assert rf["energy"] == pytest.approx(ro["energy"], abs=1e-9)
        rs = iqcc.iqcc_iterate(Hs, th, ph, w.n_gen, w.eps, w.max_terms)
        assert rs["energy"] == pytest.approx(ro["energy"], abs=1e-9)


def test_torch_caching_allocator_path():
    """Device memory from PyTorch's caching allocator through the alloc/free hooks."""
    n = 30
    _, x, z, c = synth.random_hamiltonian(n, 20_000, 12)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, torch_alloc=True)
    rng = np.random.Generator(np.random.PCG64(12))
    for _ in range(3):
        gx, gz = synth.random_generator(n, rng)
        iqcc.iqcc_dress(H, gx, gz, [0.4])
        o.dress(gx, gz, 0.4)
    iqcc.iqcc_prune(H, 1e-4)
    o.prune(1e-4)
    assert not compare(iqcc.iqcc_export(H), o.export(), eps=1e-4)
    H.close()


@pytest.mark.parametrize("cap", [150_001, 299_000, 20_000])
def test_term_limit_select_on_large_sets(cap):
    """More rows than the exact-sort bucket (65536): the 12-bit radix select
    narrows the threshold bucket first; ties at the threshold in key order."""
    n = 40
    _, x, z, c = synth.random_hamiltonian(n, 320_000, 77)
    c = np.round(c, 4)
    c[c == 0] = 1e-4
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    assert iqcc.iqcc_prune(H, 0.0, cap) == o.prune(0.0, cap)
    gx, gz, gc = iqcc.iqcc_export(H)
    ox, oz, oc = o.export()
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gc, oc)


@pytest.mark.parametrize("n", [20, 100])
def test_dress_after_compression_finds_kept_keys(n):
    """Compression rebuilds each partition of the index from its own entries
    (new rows through the compaction map, removed rows dropped); later dresses
    must find every kept key and see removed keys as absent."""
    rng = np.random.Generator(np.random.PCG64(n))
    _, x, z, c = synth.random_hamiltonian(n, 60_000, 300 + n)
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    for rnd in range(4):
        eps = float(np.quantile(np.abs(iqcc.iqcc_export(H)[2]), 0.4))
        assert iqcc.iqcc_prune(H, eps, 0) == o.prune(eps, 0)
        for _ in range(3):
            gx, gz = synth.random_generator(n, rng, weight=3)
            t = float(rng.uniform(-2, 2))
            iqcc.iqcc_dress(H, gx, gz, [t])
            o.dress(gx, gz, t)
        bad = compare(iqcc.iqcc_export(H), o.export(), eps=eps)
        assert not bad, bad[:5]
        assert len(H) == len(o)


@pytest.mark.parametrize("frac", [0.3, 0.7])
def test_holes_energy_dis_and_defragmentation(frac):
    """Compression leaves holes (removed rows stay in place until an append
    reuses them); with more than half the rows removed the library compacts
    and rebuilds its index.  Every reduction must ignore the holes."""
    n = 40
    rng = np.random.Generator(np.random.PCG64(int(frac * 100)))
    _, x, z, c = synth.random_hamiltonian(n, 150_000, 41, density=0.2)
    x[: len(x) // 4] = 0
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    th, ph = synth.qmf_angles(n, "basis")
    for rnd in range(3):
        eps = float(np.quantile(np.abs(iqcc.iqcc_export(H)[2]), frac))
        assert iqcc.iqcc_prune(H, eps, 0) == o.prune(eps, 0)
        assert len(H) == len(o)
        assert iqcc.iqcc_qmf_energy(H, th, ph) == pytest.approx(o.energy(th, ph), abs=1e-9)
        gx, gz = synth.random_generator(n, rng, weight=2)
        assert np.allclose(iqcc.iqcc_generator_abc(H, gx, gz, th, ph), o.abc(gx, gz, th, ph), rtol=0, atol=1e-9)
        ox, oz, og = o.dis(th, ph)
        hx, hz, hg = iqcc.iqcc_dis_gradients(H, th, ph)
        assert len(hg) == len(og)
        ref = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(ox, oz, og)}
        got = {(a.tobytes(), b.tobytes()): v for a, b, v in zip(hx, hz, hg)}
        assert ref.keys() == got.keys()
        for _ in range(2):
            gx, gz = synth.random_generator(n, rng, weight=3)
            t = float(rng.uniform(-2, 2))
            iqcc.iqcc_dress(H, gx, gz, [t])
            o.dress(gx, gz, t)
        bad = compare(iqcc.iqcc_export(H), o.export(), eps=eps)
        assert not bad, bad[:5]


@pytest.mark.parametrize("n", [10, 100, 200])
def test_load_of_canonical_input_and_of_sorted_input_with_repeats(n):
    """Input already in canonical order with distinct keys (an export) is loaded
    without sorting; zeros are still dropped.  Sorted input with repeated keys
    still has its repeats summed."""
    _, x, z, c = synth.random_hamiltonian(n, 20_000, 500 + n)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    ex, ez, ec = iqcc.iqcc_export(H)
    ec = ec.copy()
    ec[::7] = 0.0
    H2 = iqcc.iqcc_load_hamiltonian(n, ex, ez, ec)
    o = oracle.Oracle(n, ex, ez, ec)
    gx, gz, gc = iqcc.iqcc_export(H2)
    ox, oz, oc = o.export()
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gc, oc)
    assert len(H2) == int(np.count_nonzero(ec))
    rx = np.repeat(ex, 2, axis=0)
    rz = np.repeat(ez, 2, axis=0)
    rc = np.repeat(ec, 2) * 0.5
    H3 = iqcc.iqcc_load_hamiltonian(n, rx, rz, rc)
    o3 = oracle.Oracle(n, rx, rz, rc)
    gx, gz, gc = iqcc.iqcc_export(H3)
    ox, oz, oc = o3.export()
    assert np.array_equal(gx, ox) and np.array_equal(gz, oz) and np.array_equal(gc, oc)


def test_load_rejects_bits_above_n_qubits_in_a_large_input():
    """Inputs beyond the host-checked size are checked on the device while packed."""
    n = 40
    _, x, z, c = synth.random_hamiltonian(n, 200_000, 17)
    z = z.copy()
    z[123_456, 0] |= np.uint64(1) << np.uint64(45)
    with pytest.raises(iqcc.IqccError) as err:
        iqcc.iqcc_load_hamiltonian(n, x, z, c)
    assert err.value.status == 1


def _host(shape, dtype, pinned):
    """Zeroed host array; page-locked (torch's pinned allocator) when `pinned`."""
    if not pinned:
        return None, np.zeros(shape, dtype)
    import torch
    nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
    t = torch.zeros(max(nbytes, 8), dtype=torch.uint8, pin_memory=True)
    return t, t.numpy()[:nbytes].view(dtype).reshape(shape)


def _export_capped(H, cap, pinned=False):
    """iqcc_export with a row limit (the first `cap` rows of the canonical
    order), into pageable or page-locked host arrays."""
    import ctypes
    n = ctypes.c_int64(0)
    keep = []
    arrays = []
    for shape, dtype in (((max(cap, 1), H.W), np.uint64), ((max(cap, 1), H.W), np.uint64), ((max(cap, 1),), np.float64)):
        t, a = _host(shape, dtype, pinned)
        keep.append(t)
        arrays.append(a)
    x, z, c = arrays
    H._check(iqcc._export(H._h, cap, ctypes.byref(n), x.ctypes.data_as(iqcc._u64p), z.ctypes.data_as(iqcc._u64p),
                          c.ctypes.data_as(iqcc._f64p)))
    return n.value, x[:cap].copy(), z[:cap].copy(), c[:cap].copy()


@pytest.mark.parametrize("n", [7, 64, 100, 130, 200])
@pytest.mark.parametrize("n_gen", [0, 1, 4])
def test_export_after_dressing_sorted_prefix_and_appended_rows(n, n_gen):
    """Export of a loaded (sorted) table after 0, 1 or 4 dressings: no appended
    rows, appended rows below half of the table (sorted prefix merged with the
    sorted rest) and above half (full sort); full and row-limited exports, into
    pageable arrays (through device scratch) and page-locked ones (written by
    the device directly)."""
    rng = np.random.Generator(np.random.PCG64(700 + n + n_gen))
    _, x, z, c = synth.random_hamiltonian(n, 30_011, 800 + n, density=min(0.5, 12 / n))
    o = oracle.Oracle(n, x, z, c)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    if n_gen:
        gens = [synth.random_generator(n, rng, weight=3) for _ in range(n_gen)]
        taus = rng.uniform(-1.2, 1.2, n_gen)
        for (gx, gz), t in zip(gens, taus):
            o.dress(gx, gz, t)
        iqcc.iqcc_dress(H, np.array([g[0] for g in gens]), np.array([g[1] for g in gens]), taus)
    full = iqcc.iqcc_export(H)
    bad = compare(full, o.export())
    assert not bad, bad[:5]
    M = len(full[2])
    for pinned in (False, True):
        for cap in (1, M // 3 + 5, M - 1, M):
            m, cx, cz, cc = _export_capped(H, cap, pinned)
            assert m == M
            assert np.array_equal(cx, full[0][:cap]) and np.array_equal(cz, full[1][:cap])
            assert np.array_equal(cc, full[2][:cap])
