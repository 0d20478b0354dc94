"""Partitioned dressing on one GPU (App. B's bit-wise partitioning): a
Hamiltonian split over 2 or 4 contexts by key bits, dressed through
iqcc_cross_rows / iqcc_dress_cross for generators that flip a partition bit
and iqcc_dress otherwise, against the oracle dressing the whole H."""
import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import partitioned as pt
from paper_2603_08883_gb300 import synth
from tests.compare import compare

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)


def _masks(n, parts):
    W = (n + 63) // 64
    mx = np.zeros(W, np.uint64)
    mz = np.zeros(W, np.uint64)
    mx[0] = np.uint64(1 << 3)
    if parts == 4:
        mz[W - 1] = np.uint64(1 << ((n - 1) % 64))  # the last qubit's z bit
    return mx, mz


@pytest.mark.parametrize("n,m,seed", [(24, 20_000, 1), (100, 30_011, 2), (200, 12_007, 3)])
@pytest.mark.parametrize("parts", [2, 4])
def test_partitioned_steps_match_the_oracle(n, m, seed, parts):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, m, 100 + seed, density=min(0.5, 12 / n))
    th, ph = synth.qmf_angles(n, "uniform", seed=seed)
    mx, mz = _masks(n, parts)
    P = pt.PartitionedHamiltonian(n, x, z, c, mx, mz)
    assert len(P.parts) == parts and len(P) == len(c)
    o = oracle.Oracle(n, x, z, c)
    shifts = []
    for k in range(6):
        gx, gz = synth.random_generator(n, rng, weight=3)
        if k % 2 == 0:  # every other generator flips the first partition bit (x of qubit 3)
            gx, gz = gx.copy(), gz.copy()
            gx[0] |= np.uint64(1 << 3)
            if sum(bin(int(a & b)).count("1") for a, b in zip(gx, gz)) % 2 == 0:
                gz[0] ^= np.uint64(1 << 3)  # X <-> Y on qubit 3: keeps an odd number of Y letters
        shifts.append(pt.generator_shift(gx, gz, mx, mz))
        a, b, cc = o.abc(gx, gz, th, ph)
        pa, pb, pc = P.abc(gx, gz, th, ph)
        assert (pa, pb, pc) == pytest.approx((a, b, cc), abs=1e-10)
        tau = P.step(gx, gz, th, ph)
        o.dress(gx, gz, tau)
    assert any(s != 0 for s in shifts)
    bad = compare(P.export(), o.export())
    assert not bad, bad[:5]
    assert P.energy(th, ph) == pytest.approx(o.energy(th, ph), abs=1e-9)
    P.close()


def test_cross_rows_are_the_anticommuting_rows():
    n = 100
    rng = np.random.Generator(np.random.PCG64(9))
    _, x, z, c = synth.random_hamiltonian(n, 5000, 19, density=0.2)
    gx, gz = synth.random_generator(n, rng, weight=4)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    rx, rz, rc = iqcc.iqcc_cross_rows(H, gx, gz)
    anti = [((bin(int(a[0] & gz[0])).count("1") + bin(int(a[1] & gz[1])).count("1")
              + bin(int(b[0] & gx[0])).count("1") + bin(int(b[1] & gx[1])).count("1")) & 1) == 1
            for a, b in zip(x, z)]
    want = {(a.tobytes(), b.tobytes(), float(cc)) for a, b, cc, f in zip(x, z, c, anti) if f}
    assert {(a.tobytes(), b.tobytes(), float(cc)) for a, b, cc in zip(rx, rz, rc)} == want
    assert len(rc) == sum(anti) > 0


def test_dress_cross_errors_leave_h_unchanged():
    n = 30
    _, x, z, c = synth.random_hamiltonian(n, 400, 5, density=0.3)
    rng = np.random.Generator(np.random.PCG64(5))
    gx, gz = synth.random_generator(n, rng, weight=2)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=450)
    before = iqcc.iqcc_export(H)
    px, pz, pc = x[:100], z[:100], c[:100]
    with pytest.raises(iqcc.IqccError) as e:      # 400 + 100 rows above the capacity
        iqcc.iqcc_dress_cross(H, gx, gz, 0.3, px, pz, pc)
    assert e.value.status == 4
    bad_z = pz.copy()
    bad_z[7, 0] |= np.uint64(1 << 40)            # a bit above n_qubits
    H2 = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_dress_cross(H2, gx, gz, 0.3, px, bad_z, pc)
    assert e.value.status == 1
    for got, want in zip(iqcc.iqcc_export(H), before):
        assert np.array_equal(got, want)
    for got, want in zip(iqcc.iqcc_export(H2), before):
        assert np.array_equal(got, want)


def test_partitioned_dress_with_an_empty_side():
    """One partition empty: it sends no rows, scales nothing and appends every
    partner; the other side rotates against an empty peer set (cos(tau) only)."""
    n = 40
    rng = np.random.Generator(np.random.PCG64(12))
    _, x, z, c = synth.random_hamiltonian(n, 3000, 77, density=0.25)
    x = x.copy()
    x[:, 0] &= ~np.uint64(1 << 3)                    # every string in partition 0
    keys = np.unique(np.concatenate([x, z], 1), axis=0, return_index=True)[1]
    x, z, c = x[keys], z[keys], c[keys]
    mx, mz = _masks(n, 2)
    P = pt.PartitionedHamiltonian(n, x, z, c, mx, mz)
    assert len(P.parts[1]) == 0
    o = oracle.Oracle(n, x, z, c)
    gx, gz = synth.random_generator(n, rng, weight=3)
    gx, gz = gx.copy(), gz.copy()
    gx[0] |= np.uint64(1 << 3)
    if sum(bin(int(a & b)).count("1") for a, b in zip(gx, gz)) % 2 == 0:
        gz[0] ^= np.uint64(1 << 3)
    P.dress(gx, gz, 0.35)
    o.dress(gx, gz, 0.35)
    assert len(P.parts[1]) > 0
    bad = compare(P.export(), o.export())
    assert not bad, bad[:5]
    P.close()


@pytest.mark.parametrize("n,rows,eps,limit", [(64, 20_000, 0.0, 9000), (64, 20_000, 1e-3, 5000), (64, 20_000, 0.0, 3),
                                              (100, 200_000, 0.0, 120_000), (200, 200_000, 1e-3, 70_001)])
def test_partitioned_term_limit_matches_the_oracle(n, rows, eps, limit):
    """The term limit over the whole split Hamiltonian (iqcc_prune_parts:
    threshold from every part's coefficients, ties in canonical order across
    parts) against the oracle's compression of the unsplit one; coefficients
    rounded to create ties at the threshold.  The 200,000-row cases need
    several 12-bit select passes before the threshold bucket is small."""
    rng = np.random.Generator(np.random.PCG64(31 + n))
    _, x, z, c = synth.random_hamiltonian(n, rows, 91 + n, density=0.2)
    c = np.round(c, 2)
    keep = c != 0
    x, z, c = x[keep], z[keep], c[keep]
    mx, mz = _masks(n, 4)
    P = pt.PartitionedHamiltonian(n, x, z, c, mx, mz)
    assert min(len(H) for H in P.parts) > 0
    o = oracle.Oracle(n, x, z, c)
    removed = P.prune(eps, limit)
    assert removed == o.prune(eps, limit)
    bad = compare(P.export(), o.export())
    assert not bad, bad[:5]
    P.close()


def test_dress_pair_matches_the_host_exchange_and_errors_leave_both_unchanged():
    """iqcc_dress_pair (both partitions' anticommuting rows in one set of bins
    on the device) against the host exchange (iqcc_cross_rows, then
    iqcc_dress_cross on each side) and the oracle, for a generator that flips
    the partition bit; then its argument and capacity errors."""
    n = 100
    rng = np.random.Generator(np.random.PCG64(41))
    _, x, z, c = synth.random_hamiltonian(n, 40_000, 43, density=0.12)
    mx, mz = _masks(n, 2)
    gx, gz = synth.random_generator(n, rng, weight=3)
    gx, gz = gx.copy(), gz.copy()
    gx[0] |= np.uint64(1 << 3)
    if sum(bin(int(a & b)).count("1") for a, b in zip(gx, gz)) % 2 == 0:
        gz[0] ^= np.uint64(1 << 3)
    assert pt.generator_shift(gx, gz, mx, mz) == 1
    tau = 0.37
    P = pt.PartitionedHamiltonian(n, x, z, c, mx, mz)
    P.dress(gx, gz, tau)                                 # the device pair dress
    Q = pt.PartitionedHamiltonian(n, x, z, c, mx, mz)    # the host exchange
    sent = [iqcc.iqcc_cross_rows(H, gx, gz) for H in Q.parts]
    for a, H in enumerate(Q.parts):
        iqcc.iqcc_dress_cross(H, gx, gz, tau, *sent[a ^ 1])
    o = oracle.Oracle(n, x, z, c)
    o.dress(gx, gz, tau)
    for got in (P.export(), Q.export()):
        bad = compare(got, o.export())
        assert not bad, bad[:5]
    for a in (0, 1):                                     # every row landed in the partition owning it
        assert np.all(pt.partition_of(*iqcc.iqcc_export(P.parts[a])[:2], mx, mz) == a)
    ax, az = P.pattern(0)
    with pytest.raises(iqcc.IqccError) as e:             # the same context twice
        iqcc.iqcc_dress_pair(P.parts[0], P.parts[0], gx, gz, tau, mx, mz, ax, az)
    assert e.value.status == 1
    bad_ax = ax.copy()
    bad_ax[1] |= np.uint64(1)                           # a bit outside the masks
    with pytest.raises(iqcc.IqccError) as e:
        iqcc.iqcc_dress_pair(P.parts[0], P.parts[1], gx, gz, tau, mx, mz, bad_ax, az)
    assert e.value.status == 1
    part = pt.partition_of(x, z, mx, mz)
    A = iqcc.iqcc_load_hamiltonian(n, x[part == 0], z[part == 0], c[part == 0], capacity=int(np.sum(part == 0)) + 1)
    B = iqcc.iqcc_load_hamiltonian(n, x[part == 1], z[part == 1], c[part == 1])
    before = [iqcc.iqcc_export(A), iqcc.iqcc_export(B)]
    with pytest.raises(iqcc.IqccError) as e:             # A could receive a partner per row of B
        iqcc.iqcc_dress_pair(A, B, gx, gz, tau, mx, mz, ax, az)
    assert e.value.status == 4
    for H, want in zip((A, B), before):
        for got, w in zip(iqcc.iqcc_export(H), want):
            assert np.array_equal(got, w)
    for H in (A, B):
        H.close()
    P.close()
    Q.close()
