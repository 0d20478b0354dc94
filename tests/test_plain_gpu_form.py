"""The plain PyTorch-tensor form (the same-GPU comparison in bench.py) against
the oracle: dress, merge, prune, energy and A, B, C on seeded inputs.  On the
CPU here (it is plain tensor code); on the GPU under the gpu marker."""
import math

import numpy as np
import pytest

import oracle
from baseline.plain_gpu import PlainHamiltonian, popcount
from paper_2603_08883_gb300 import synth
from tests.compare import compare

torch = pytest.importorskip("torch")


def test_popcount_matches_python():
    rng = np.random.Generator(np.random.PCG64(1))
    v = rng.integers(0, 2**64, 1000, dtype=np.uint64)
    v[:4] = [0, 2**64 - 1, 2**63, 1]
    got = popcount(torch.from_numpy(v.view(np.int64))).numpy()
    assert list(got) == [bin(int(a)).count("1") for a in v]


def _run(n, m, seed, device, n_gen=3, eps=0.0):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, m, seed, density=min(0.5, 10 / n))
    th, ph = synth.qmf_angles(n, "uniform", seed=seed)
    o = oracle.Oracle(n, x, z, c)
    p = PlainHamiltonian(n, x, z, c, device=device)
    for _ in range(n_gen):
        gx, gz = synth.random_generator(n, rng, weight=3)
        a, b, cc = p.abc(gx, gz, th, ph)
        oa, ob, oc = o.abc(gx, gz, th, ph)
        assert a == pytest.approx(oa, abs=1e-10) and b == pytest.approx(ob, abs=1e-10)
        assert cc == pytest.approx(oc, abs=1e-10)
        tau = math.atan2(-oc, -ob) if (ob or oc) else 0.0
        p.dress(gx, gz, tau)
        o.dress(gx, gz, tau)
    if eps:
        assert p.prune(eps) == o.prune(eps)
    bad = compare(p.export(), o.export(), eps=eps)
    assert not bad, bad[:5]
    assert p.energy(th, ph) == pytest.approx(o.energy(th, ph), abs=1e-9)


@pytest.mark.parametrize("n,m,seed", [(1, 3, 1), (8, 300, 2), (24, 2000, 3), (100, 3000, 4), (130, 1500, 5)])
def test_plain_form_matches_oracle_on_cpu(n, m, seed):
    _run(n, m, seed, "cpu")


def test_plain_form_prunes_like_the_oracle():
    _run(24, 3000, 9, "cpu", n_gen=4, eps=1e-3)


@pytest.mark.gpu
@pytest.mark.parametrize("n,m,seed", [(24, 20_000, 6), (100, 20_000, 7), (200, 8000, 8)])
def test_plain_form_matches_oracle_on_gpu(n, m, seed):
    _run(n, m, seed, "cuda")
