"""Load of rows in any order (repeated strings summed by partition and join,
or by the sort when one string repeats thousands of times) and the unordered
export, against the oracle.  Repeated strings are summed in input order on
both sides, so the coefficients agree bit for bit."""
import numpy as np
import pytest

from paper_2603_08883_gb300 import synth

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)
import oracle  # noqa: E402

pytestmark = pytest.mark.gpu


def _exact(gpu, ref):
    for a, b in zip(gpu, ref):
        assert a.shape == b.shape
        assert np.array_equal(a, b)


def _with_repeats(n, m, seed, copies):
    """m distinct random strings, some repeated (up to `copies` times, with
    exact cancellations among them), shuffled."""
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, m, seed, density=0.2)
    rep = rng.choice(len(c), len(c) // 5, replace=False)
    xs, zs, cs = [x], [z], [c]
    for k in range(1, copies):
        sel = rep[: len(rep) // k]
        xs.append(x[sel])
        zs.append(z[sel])
        cs.append(np.where(rng.random(len(sel)) < 0.3, -c[sel], rng.normal(size=len(sel))))
    x, z, c = np.concatenate(xs), np.concatenate(zs), np.concatenate(cs)
    perm = rng.permutation(len(c))
    return x[perm], z[perm], c[perm]


@pytest.mark.parametrize("n,m,copies", [(24, 50_000, 3), (100, 300_000, 4), (200, 80_000, 5)])
def test_load_in_any_order_matches_the_oracle(n, m, copies):
    x, z, c = _with_repeats(n, m, 7 + n, copies)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    assert len(H) == len(o)
    _exact(iqcc.iqcc_export(H), o.export())
    H.close()


def test_many_copies_of_one_string_are_summed_in_input_order():
    """10,000 copies of one string overflow a join block: the load sorts."""
    n = 64
    x, z, c = _with_repeats(n, 20_000, 5, 2)
    rng = np.random.Generator(np.random.PCG64(3))
    k = 10_000
    x = np.concatenate([x, np.repeat(x[:1], k, 0)])
    z = np.concatenate([z, np.repeat(z[:1], k, 0)])
    c = np.concatenate([c, rng.normal(size=k)])
    perm = rng.permutation(len(c))
    x, z, c = x[perm], z[perm], c[perm]
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    _exact(iqcc.iqcc_export(H), o.export())
    H.close()


def test_unordered_export_round_trip():
    """iqcc_export_rows holds the same strings as iqcc_export; loading it back
    gives the same Hamiltonian; a dressed H (rows in bin order) too."""
    n = 100
    _, x, z, c = synth.random_hamiltonian(n, 120_000, 11, density=0.15)
    rng = np.random.Generator(np.random.PCG64(11))
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    gx, gz = synth.random_generator(n, rng, weight=3)
    iqcc.iqcc_dress(H, gx.reshape(1, -1), gz.reshape(1, -1), [0.3])
    ref = iqcc.iqcc_export(H)
    rx, rz, rc = iqcc.iqcc_export_rows(H)
    assert len(rc) == len(ref[2])
    keys = np.lexsort([rz[:, w] for w in range(rz.shape[1])] + [rx[:, w] for w in range(rx.shape[1])])
    _exact((rx[keys], rz[keys], rc[keys]), ref)
    H2 = iqcc.iqcc_load_hamiltonian(n, rx, rz, rc)
    _exact(iqcc.iqcc_export(H2), ref)
    H.close()
    H2.close()
