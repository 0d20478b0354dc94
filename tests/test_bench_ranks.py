"""Host logic of bench.py's multi-rank (replicas) path on two CPU ranks over gloo."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench
    from paper_2603_08883_gb300 import synth
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.25][rank]
        units = [1e9, 3e9][rank]
        t, u = bench.reduce_over_ranks(dist, seconds, units, "cpu")
        w = bench.workload_for_rank(synth.WORKLOADS["jw8"], rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, w.seed)
        q.put((rank, t, u, seeds))
    finally:
        dist.destroy_process_group()


def test_replica_timing_is_max_over_ranks_and_units_are_summed():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, u, seeds in res:
        assert t == 2.25 and u == 4e9
        assert seeds[0] != seeds[1]


def test_single_rank_is_identity():
    import bench
    from paper_2603_08883_gb300 import synth
    assert bench.reduce_over_ranks(None, 3.0, 7.0, "cpu") == (3.0, 7.0)
    w = synth.WORKLOADS["jw100"]
    assert bench.workload_for_rank(w, 0) is w
