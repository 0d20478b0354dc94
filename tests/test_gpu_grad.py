"""Adjoint of the dressed QMF energy on the GPU (iqcc_energy_gradients and the
torch.autograd binding) against the oracle's derivatives (dress a copy, then
differentiate every string qubit by qubit) and against finite differences."""
import numpy as np
import pytest

import oracle
from paper_2603_08883_gb300 import synth

pytestmark = pytest.mark.gpu

iqcc = pytest.importorskip("paper_2603_08883_gb300.iqcc", exc_type=ImportError)
torch = pytest.importorskip("torch")


def _angles(n, kind, rng):
    if kind == "basis":
        return np.where(np.arange(n) < n // 2, np.pi, 0.0), np.zeros(n)
    return rng.uniform(0, np.pi, n), rng.uniform(0, 2 * np.pi, n)


def _close(got, ref, scale, rel=1e-10):
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    return np.all(np.abs(got - ref) <= rel * np.abs(ref) + 1e-13 * scale), np.max(np.abs(got - ref))


@pytest.mark.parametrize("n", [5, 8, 24, 64, 65, 100, 130, 200])
@pytest.mark.parametrize("kind", ["general", "basis"])
@pytest.mark.parametrize("with_gen", [False, True])
def test_energy_gradients_match_oracle(n, kind, with_gen):
    rng = np.random.Generator(np.random.PCG64(1000 * n + 10 * (kind == "basis") + with_gen))
    m = 3000 if n <= 100 else 1500
    _, x, z, c = synth.random_hamiltonian(n, m, 7000 + n, density=min(0.5, 12.0 / n))
    theta, phi = _angles(n, kind, rng)
    gx = gz = None
    tau = 0.0
    if with_gen:
        gx, gz = synth.random_generator(n, rng, weight=3)
        tau = float(rng.uniform(-1.2, 1.2))
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    e, dt, dp, dtau = iqcc.iqcc_energy_gradients(H, theta, phi, gx, gz, tau)
    oe, odt, odp, odtau = o.energy_gradients(theta, phi, gx, gz, tau)
    scale = float(np.abs(c).sum())
    for got, ref in ((e, oe), (dt, odt), (dp, odp), (dtau, odtau)):
        ok, worst = _close(got, ref, scale)
        assert ok, worst
    if not with_gen:
        assert e == pytest.approx(iqcc.iqcc_qmf_energy(H, theta, phi), rel=1e-12, abs=1e-13 * scale)
    else:
        a, b, cc = iqcc.iqcc_generator_abc(H, gx, gz, theta, phi)
        assert e == pytest.approx(a + b * np.cos(tau) + cc * np.sin(tau), rel=1e-12, abs=1e-13 * scale)


def _chain_hamiltonian(n, m, rng):
    """Jordan-Wigner-like strings: X or Y at p < q and Z on every qubit between
    (runs of Z letters, many crossing the 64-qubit word boundary), some with a
    second chain, plus random strings."""
    W = (n + 63) // 64
    xs, zs = [], []
    for _ in range(m):
        xb = np.zeros(n, bool)
        zb = np.zeros(n, bool)
        for _ in range(int(rng.integers(1, 3))):
            p, q = sorted(rng.choice(n, 2, replace=False))
            zb[p + 1:q] ^= True
            for k in (p, q):
                xb[k] = True
                zb[k] = bool(rng.integers(0, 2))
        xs.append(xb)
        zs.append(zb)
    pack = lambda b: np.array([[int("".join("1" if v else "0" for v in row[64 * w:64 * w + 64][::-1]) or "0", 2)
                                for w in range(W)] for row in b], np.uint64)
    x, z = pack(np.array(xs)), pack(np.array(zs))
    keys = np.unique(np.concatenate([x, z], 1), axis=0)
    c = rng.standard_normal(len(keys))
    return keys[:, :W].copy(), keys[:, W:].copy(), c


@pytest.mark.parametrize("n", [70, 100, 200])
@pytest.mark.parametrize("with_gen", [False, True])
def test_energy_gradients_of_z_chains_at_general_angles(n, with_gen):
    """Long Z runs take the run-difference sums of the general path; runs
    that cross a word boundary included."""
    rng = np.random.Generator(np.random.PCG64(500 + n + with_gen))
    x, z, c = _chain_hamiltonian(n, 2000, rng)
    theta, phi = _angles(n, "general", rng)
    gx = gz = None
    tau = 0.0
    if with_gen:
        gx, gz = synth.random_generator(n, rng, weight=3)
        tau = 0.7
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    o = oracle.Oracle(n, x, z, c)
    got = iqcc.iqcc_energy_gradients(H, theta, phi, gx, gz, tau)
    ref = o.energy_gradients(theta, phi, gx, gz, tau)
    scale = float(np.abs(c).sum())
    for g, r in zip(got, ref):
        ok, worst = _close(g, r, scale)
        assert ok, worst


def test_energy_gradients_edge_cases():
    n = 6
    # identity only: constant energy, zero gradient
    x = np.zeros((1, 1), np.uint64)
    H = iqcc.iqcc_load_hamiltonian(n, x, x, np.array([2.5]))
    e, dt, dp, dtau = iqcc.iqcc_energy_gradients(H, np.full(n, 0.3), np.full(n, 0.2))
    assert e == 2.5 and not dt.any() and not dp.any() and dtau == 0.0
    # everything pruned away: all zero
    _, x, z, c = synth.random_hamiltonian(n, 50, 3)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    iqcc.iqcc_prune(H, 1e9, 0)
    assert len(H) == 0
    e, dt, dp, dtau = iqcc.iqcc_energy_gradients(H, np.full(n, 0.3), np.full(n, 0.2), np.array([1], np.uint64),
                                                 np.array([0], np.uint64), 0.4)
    assert e == 0.0 and not dt.any() and not dp.any() and dtau == 0.0
    # argument errors
    with pytest.raises(ValueError):
        iqcc.iqcc_energy_gradients(H, np.zeros(n), np.zeros(n), np.array([1], np.uint64), None)
    H2 = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    with pytest.raises(iqcc.IqccError) as err:
        iqcc.iqcc_energy_gradients(H2, np.zeros(n), np.zeros(n), np.array([1 << 7], np.uint64),
                                   np.array([0], np.uint64), 0.1)
    assert err.value.status == 1


def test_autograd_matches_finite_differences_and_optimises():
    """torch.autograd.gradcheck through the adjoint kernel (8-qubit workload,
    one generator), then a few L-BFGS steps on the angles and the amplitude:
    the energy falls and agrees with the oracle at the final parameters."""
    from paper_2603_08883_gb300.autograd import dressed_energy
    w = synth.WORKLOADS["jw8"]
    n, x, z, c = synth.workload_hamiltonian(w)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    rng = np.random.Generator(np.random.PCG64(5))
    th0, ph0 = synth.qmf_angles(n, "uniform", seed=w.seed)
    gx, gz = synth.random_generator(n, rng, weight=2)
    theta = torch.tensor(th0, dtype=torch.float64, requires_grad=True)
    phi = torch.tensor(ph0, dtype=torch.float64, requires_grad=True)
    tau = torch.tensor(0.3, dtype=torch.float64, requires_grad=True)
    f = lambda t, p, a: dressed_energy(H, t, p, a, gx, gz)
    assert torch.autograd.gradcheck(f, (theta, phi, tau), eps=1e-6, atol=1e-6, rtol=1e-5)
    opt = torch.optim.LBFGS([theta, phi, tau], max_iter=30, line_search_fn="strong_wolfe")
    e0 = float(f(theta, phi, tau).detach())

    def closure():
        opt.zero_grad()
        e = f(theta, phi, tau)
        e.backward()
        return e
    opt.step(closure)
    e1 = float(f(theta, phi, tau).detach())
    assert e1 < e0 - 1e-3
    o = oracle.Oracle(n, x, z, c)
    oe, _, _, _ = o.energy_gradients(theta.detach().numpy(), phi.detach().numpy(), gx, gz, float(tau.detach()))
    assert e1 == pytest.approx(oe, abs=1e-10)
