"""Host logic of the partitioned dress (App. B's bit-wise partitioning): the
partition of a key, the generator's partition offset, and the exchange step
between ranks over gloo on the CPU.  Each rank holds one partition in a plain
dictionary engine written here from the partition rule; the union of the
parts after every step is checked against the oracle dressing the whole H."""
import math
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from paper_2603_08883_gb300 import partitioned as pt
from paper_2603_08883_gb300 import synth
from tests.compare import compare


def _popc(v):
    return bin(int(v)).count("1")


def _popc_and(a, b):
    return sum(_popc(int(u) & int(v)) for u, v in zip(a, b))


class DictEngine:
    """One partition as {(x, z): c}; the exchange's four steps by their definition."""

    def __init__(self, n, x, z, c):
        self.n = n
        self.d = {(tuple(int(v) for v in a), tuple(int(v) for v in b)): float(cc) for a, b, cc in zip(x, z, c)}

    def arrays(self):
        W = (self.n + 63) // 64
        keys = list(self.d)
        x = np.array([k[0] for k in keys], np.uint64).reshape(-1, W)
        z = np.array([k[1] for k in keys], np.uint64).reshape(-1, W)
        return x, z, np.array([self.d[k] for k in keys])

    @staticmethod
    def _anti(k, gx, gz):
        return (_popc_and(k[0], gz) + _popc_and(k[1], gx)) & 1

    @staticmethod
    def _sign(t, gx, gz, q):
        """s with i T P = s P(q), q = T xor P."""
        e = (_popc_and(t[0], t[1]) + _popc_and(gx, gz) + 2 * _popc_and(t[1], gx) - _popc_and(q[0], q[1])) % 4
        return 1.0 if e == 3 else -1.0

    def cross_rows(self, gx, gz):
        W = (self.n + 63) // 64
        rows = [(k, c) for k, c in self.d.items() if self._anti(k, gx, gz)]
        x = np.array([k[0] for k, _ in rows], np.uint64).reshape(-1, W)
        z = np.array([k[1] for k, _ in rows], np.uint64).reshape(-1, W)
        return x, z, np.array([c for _, c in rows])

    def dress_cross(self, gx, gz, tau, px, pz, pc):
        peer = {(tuple(int(v) for v in a), tuple(int(v) for v in b)): float(c) for a, b, c in zip(px, pz, pc)}
        flip = lambda k: (tuple(int(a) ^ int(g) for a, g in zip(k[0], gx)),
                          tuple(int(b) ^ int(g) for b, g in zip(k[1], gz)))
        new = dict(self.d)
        for k, c in self.d.items():
            if not self._anti(k, gx, gz):
                continue
            t = flip(k)
            new[k] = c * math.cos(tau) + (self._sign(t, gx, gz, k) * peer[t] * math.sin(tau) if t in peer else 0.0)
        for t, c in peer.items():
            k = flip(t)
            if k not in self.d:
                new[k] = self._sign(t, gx, gz, k) * c * math.sin(tau)
        self.d = new

    def dress(self, gx, gz, tau):
        o = oracle.Oracle(self.n, *self.arrays())
        o.dress(gx, gz, tau)
        self.d = DictEngine(self.n, *o.export()).d

    def abc(self, gx, gz, theta, phi):
        return oracle.Oracle(self.n, *self.arrays()).abc(gx, gz, theta, phi)


def test_partition_index_and_generator_offset():
    W = 2
    x = np.array([[0, 0], [1 << 3, 0], [0, 1 << 5], [1 << 3, 1 << 5]], np.uint64)
    z = np.array([[1 << 7, 0], [0, 0], [1 << 7, 0], [0, 0]], np.uint64)
    mx = np.array([1 << 3, 1 << 5], np.uint64)
    mz = np.array([1 << 7, 0], np.uint64)
    assert list(pt.partition_of(x, z, mx, mz)) == [4, 1, 6, 3]
    assert pt.generator_shift(np.array([1 << 3, 0], np.uint64), np.zeros(W, np.uint64), mx, mz) == 1
    assert pt.generator_shift(np.array([0, 1 << 9], np.uint64), np.array([1, 0], np.uint64), mx, mz) == 0
    # the partner of a key lies at the key's partition xor the generator's offset
    rng = np.random.Generator(np.random.PCG64(2))
    for _ in range(50):
        kx, kz, gx, gz = (rng.integers(0, 2**63, (1, W), dtype=np.uint64) for _ in range(4))
        a = pt.partition_of(kx, kz, mx, mz)[0]
        b = pt.partition_of(kx ^ gx, kz ^ gz, mx, mz)[0]
        assert b == a ^ pt.generator_shift(gx, gz, mx, mz)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(n, m, seed, n_gen):
    rng = np.random.Generator(np.random.PCG64(seed))
    _, x, z, c = synth.random_hamiltonian(n, m, seed, density=min(0.5, 8 / n))
    th, ph = synth.qmf_angles(n, "uniform", seed=seed)
    gens = [synth.random_generator(n, rng, weight=3) for _ in range(n_gen)]
    return x, z, c, th, ph, gens


def _rank(rank, world, port, n, m, seed, n_gen, mx, mz, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        x, z, c, th, ph, gens = _problem(n, m, seed, n_gen)
        sel = pt.partition_of(x, z, mx, mz) == rank
        eng = DictEngine(n, x[sel], z[sel], c[sel])
        taus, shifts = [], []
        for gx, gz in gens:
            tau = pt.reduced_tau(eng, dist, gx, gz, th, ph)
            pt.exchange_dress(eng, dist, rank, gx, gz, tau, mx, mz)
            taus.append(tau)
            shifts.append(pt.generator_shift(gx, gz, mx, mz))
        q.put((rank, eng.arrays(), taus, shifts))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,mask", [(2, "x3"), (4, "x3z5")])
def test_exchange_over_gloo_matches_the_oracle_on_the_whole_hamiltonian(world, mask):
    n, m, seed, n_gen = 16, 600, 41, 8
    mx = np.array([1 << 3], np.uint64)
    mz = np.array([1 << 5 if mask == "x3z5" else 0], np.uint64)
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, n, m, seed, n_gen, mx, mz, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(world)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    taus, shifts = res[0][2], res[0][3]
    assert all(r[2] == taus for r in res)                # every rank took the same amplitudes
    assert any(s != 0 for s in shifts) and any(s == 0 for s in shifts)  # exchanges and local dresses
    x, z, c, th, ph, gens = _problem(n, m, seed, n_gen)
    o = oracle.Oracle(n, x, z, c)
    for (gx, gz), tau in zip(gens, taus):
        a, b, cc = o.abc(gx, gz, th, ph)
        assert tau == pytest.approx(pt.closed_form_tau(a, b, cc), abs=1e-9)
        o.dress(gx, gz, tau)
    union = tuple(np.concatenate([r[1][i] for r in res]) for i in range(3))
    bad = compare(union, o.export())
    assert not bad, bad[:5]


def _rank_empty_side(rank, world, port, q):
    """Partition 1 starts empty: it sends no rows and receives every partner it must append."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        n = 6
        mx = np.array([1 << 0], np.uint64)
        mz = np.array([0], np.uint64)
        x = np.array([[0], [2], [4]], np.uint64)          # all with x bit 0 clear: partition 0
        z = np.array([[1], [3], [0]], np.uint64)
        c = np.array([0.5, -1.25, 2.0])
        sel = pt.partition_of(x, z, mx, mz) == rank
        eng = DictEngine(n, x[sel], z[sel], c[sel])
        gx, gz = np.array([1], np.uint64), np.array([1], np.uint64)  # Y on qubit 0: flips partition bit 0
        pt.exchange_dress(eng, dist, rank, gx, gz, 0.4, mx, mz)
        q.put((rank, eng.arrays()))
    finally:
        dist.destroy_process_group()


def test_exchange_with_an_empty_partition():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_empty_side, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=120) for _ in range(2)), key=lambda r: r[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    x = np.array([[0], [2], [4]], np.uint64)
    z = np.array([[1], [3], [0]], np.uint64)
    c = np.array([0.5, -1.25, 2.0])
    o = oracle.Oracle(6, x, z, c)
    o.dress(np.array([1], np.uint64), np.array([1], np.uint64), 0.4)
    union = tuple(np.concatenate([r[1][i] for r in res]) for i in range(3))
    assert len(res[1][1][2]) > 0                        # the empty side received and appended partners
    bad = compare(union, o.export())
    assert not bad, bad[:5]


@pytest.mark.parametrize("n,parts", [(24, 2), (100, 4), (200, 4)])
def test_partition_pattern_round_trip(n, parts):
    """The key bits a partition is given under the masks (the owner rule of
    the two-partition dress) map back to that partition, and generator shifts
    combine partitions by xor."""
    W = (n + 63) // 64
    mx = np.zeros(W, np.uint64)
    mz = np.zeros(W, np.uint64)
    mx[0] = np.uint64(1 << 3)
    if parts == 4:
        mz[W - 1] = np.uint64(1 << ((n - 1) % 64))
    P = object.__new__(pt.PartitionedHamiltonian)   # the bookkeeping only: no contexts
    P.n, P.W, P.mx, P.mz = n, W, mx, mz
    for a in range(parts):
        px, pz = P.pattern(a)
        assert np.all((px & ~mx) == 0) and np.all((pz & ~mz) == 0)
        assert pt.partition_of(px.reshape(1, -1), pz.reshape(1, -1), mx, mz)[0] == a
        for d in range(parts):
            gx, gz = P.pattern(d)
            assert pt.generator_shift(gx, gz, mx, mz) == d
            qx, qz = px ^ gx, pz ^ gz
            assert pt.partition_of(qx.reshape(1, -1), qz.reshape(1, -1), mx, mz)[0] == a ^ d
