#!/usr/bin/env python3
"""Benchmark of the iQCC dressing path on GB300.

One step = one iQCC iteration (App. A steps 1-5) of the 100-qubit workload:
DIS screening, 8 x (A, B, C; dress; term limit), compression, energy.  The run
is the workload's own iteration sequence: W warm-up iterations, then K timed
ones on the Hamiltonian those produced, all resident in HBM.

Metric: dressed Pauli terms per second = sum over the timed iterations of M at
each generator's dress, divided by the device time of those iterations (max
over ranks).  N > 1 ranks run independent seeded Hamiltonians (weak scaling;
the path has no cross-rank exchange in this configuration).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpu|reference]
"""
from __future__ import annotations

import argparse
import faulthandler
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024
METRIC = "dressed Pauli terms/s, 100-qubit iQCC iteration"
UNIT = "terms/s"
# strings of the 100-qubit workload the oracle runs on per step (the reference arm and cpu_baseline);
# fewer than about 4000 give no DIS candidate, hence nothing to dress
REFERENCE_ROWS = 8000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpu", "reference"], default="gpu")
    ap.add_argument("--workload", default="jw100")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--max-terms", type=int, default=0,
                    help="profiling case: a lower term limit than the workload's (capacity twice it); the line "
                         "then measures that smaller configuration and says so in its config")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the measurements of the adjoint pass, learned screening, sort-based dress and batches")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(w, extra):
    cfg = {"workload": f"{w.name}: {w.notes}", "n_qubits": w.n_qubits, "orbitals": w.norb, "integrals": w.integrals,
           "reference_state": w.angles, "generators_per_iteration": w.n_gen, "eps": w.eps,
           "max_terms": w.max_terms, "capacity_rows": w.capacity, "seed": w.seed}
    cfg.update(extra)
    return cfg


def oracle_dressed(w, n, x, z, c, th, ph, rows):
    """Dressed-term count of one oracle iteration on the sample (same
    definition as the GPU metric) and its wall time."""
    import oracle
    o = oracle.Oracle(n, x[:rows], z[:rows], c[:rows])
    t0 = time.perf_counter()
    cx, cz, g = o.dis(th, ph)
    sel = [i for i in range(len(g)) if abs(g[i]) > 1e-12][: w.n_gen]
    dressed = 0
    for i in sel:
        a, b, cc = o.abc(cx[i], cz[i], th, ph)
        tau = 0.0 if (b == 0.0 and cc == 0.0) else float(np.arctan2(-cc, -b))
        dressed += len(o)
        o.dress(cx[i], cz[i], tau)
        if w.max_terms > 0 and len(o) > w.max_terms:
            o.prune(0.0, w.max_terms)
    o.prune(w.eps, w.max_terms)
    o.energy(th, ph)
    return dressed, time.perf_counter() - t0


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "out", "").splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def workload_for_rank(w, rank: int):
    """Replicas: rank r runs the workload with seed + 1000 r (an independent
    Hamiltonian of the same recipe and size)."""
    import dataclasses
    return dataclasses.replace(w, seed=w.seed + 1000 * rank) if rank else w


def reduce_over_ranks(dist, seconds: float, units: float, device):
    """(max over ranks of the timed seconds, sum over ranks of the units):
    whole-job throughput = units / seconds."""
    if dist is None:
        return seconds, units
    import torch
    tt = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    uu = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(uu, op=dist.ReduceOp.SUM)
    return float(tt.item()), float(uu.item())


def measure_adjoint(iqcc, H, n, th, ph, stream):
    """iqcc_energy_gradients on H as it stands (CUDA events around the call),
    at the workload's angles and at random general angles, with the top DIS
    candidate as generator.  Algorithmic bytes: (16W + 8) per term."""
    import torch
    M = len(H)
    W = (n + 63) // 64
    cx, cz, _ = iqcc.iqcc_dis_gradients(H, th, ph, cap=1)
    rng = np.random.Generator(np.random.PCG64(11))
    general = (rng.uniform(0, np.pi, n), rng.uniform(0, 2 * np.pi, n))
    out = {"M": M, "bytes_per_term": 16 * W + 8, "generator": "top DIS candidate, tau = 0.1"}
    peak, _ = measured_peak()
    for name, (t, p) in (("workload_angles", (th, ph)), ("general_angles", general)):
        iqcc.iqcc_energy_gradients(H, t, p, cx[0], cz[0], 0.1)  # warm-up
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        iqcc.iqcc_energy_gradients(H, t, p, cx[0], cz[0], 0.1)
        ev1.record(stream)
        ev1.synchronize()
        ms = ev0.elapsed_time(ev1)
        gbs = M * (16 * W + 8) / (ms / 1e3) / 1e9
        out[name] = {"ms": round(ms, 2), "achieved_GBs": round(gbs, 1), "frac_hbm": round(gbs / peak, 4)}
    return out


def measure_joint_optimisation(iqcc, H, th, ph, max_iter=8):
    """Joint optimisation of the QMF angles and one amplitude on H as it
    stands: L-BFGS (strong Wolfe) on E(theta, phi, tau) with the top DIS
    candidate as generator and tau = 0 to start; every evaluation is one
    adjoint pass (energy and all gradients).  Two starts: the workload's
    basis angles (every string flips an even number of qubits, so the angle
    gradients vanish there and only tau moves), and those angles with seeded
    N(0, 0.05) noise (general angles: all 2n + 1 variables move)."""
    import torch
    from paper_2603_08883_gb300.autograd import dressed_energy
    cx, cz, _ = iqcc.iqcc_dis_gradients(H, th, ph, cap=1)
    rng = np.random.Generator(np.random.PCG64(21))
    n = len(th)
    out = {"M": len(H), "generator": "top DIS candidate", "optimiser": f"L-BFGS, strong Wolfe, max_iter {max_iter}"}
    for name, (t0_, p0_) in (("basis_start", (th, ph)),
                             ("perturbed_start", (th + rng.normal(0, 0.05, n), ph + rng.normal(0, 0.05, n)))):
        theta = torch.tensor(t0_, dtype=torch.float64, requires_grad=True)
        phi = torch.tensor(p0_, dtype=torch.float64, requires_grad=True)
        tau = torch.tensor(0.0, dtype=torch.float64, requires_grad=True)
        f = lambda: dressed_energy(H, theta, phi, tau, cx[0], cz[0])
        e0 = float(f().detach())
        opt = torch.optim.LBFGS([theta, phi, tau], max_iter=max_iter, line_search_fn="strong_wolfe")
        evals = [0]

        def closure():
            opt.zero_grad()
            e = f()
            e.backward()
            evals[0] += 1
            return e
        t0 = time.perf_counter()
        opt.step(closure)
        dt = time.perf_counter() - t0
        e1 = float(f().detach())
        out[name] = {"energy_start": e0, "energy_end": e1, "tau_end": float(tau.detach()),
                     "max_angle_change": float(max((theta.detach() - torch.tensor(t0_)).abs().max(),
                                                   (phi.detach() - torch.tensor(p0_)).abs().max())),
                     "evaluations": evals[0], "s": round(dt, 2),
                     "ms_per_evaluation": round(dt / max(evals[0], 1) * 1e3, 1)}
    return out


def measure_screening(iqcc, H, th, ph):
    """The learned-screening perceptron (tensor cores, mma.sync BF16 / FP32)
    scoring every term of H as it stands: 2 (8 x 256 + 256 x 256 + 256) =
    135,680 algorithmic FLOP per term; device time from the library's events."""
    from paper_2603_08883_gb300.screening import load_model
    M = len(H)
    iqcc.iqcc_set_screening_model(H, *load_model())
    gx, gz, _ = iqcc.iqcc_dis_gradients(H, th, ph, cap=4)
    iqcc.iqcc_prune_learned(H, 0.0, M, th, ph, gx, gz)      # warm-up; a limit of M removes nothing
    before = iqcc.iqcc_get_stats(H)
    iqcc.iqcc_prune_learned(H, 0.0, M, th, ph, gx, gz)
    after = iqcc.iqcc_get_stats(H)
    ms = after["screen_ms"] - before["screen_ms"]
    terms = after["screen_terms"] - before["screen_terms"]
    flop = 135680.0 * terms
    peak = measured_peak_tensor()
    tf = flop / (ms / 1e3) / 1e12
    return {"kernel": "k_mlp_score (features + 8-256-256-1 perceptron, mma.sync m16n8k16 bf16)", "terms": terms,
            "ms": round(ms, 2), "achieved_tflops": round(tf, 1), "peak_tflops": peak[0], "peak_kind": peak[1],
            "frac": round(tf / peak[0], 4) if peak[0] else None}


def measured_peak_tensor():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured burst bf16 (MEASURED_PEAKS.json bf16_tflops)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback 1.9 PFLOP/s bf16"


def measure_sort_variant(iqcc, n, x, z, c, th, ph, stream, n_gen=8, tau=0.1):
    """The hash dress against the sort-based dress (one sort per generator, and
    all generators fused into one expansion and one sort) on the loaded
    Hamiltonian, with its top DIS candidates as generators; CUDA events around
    each API call (index upkeep included on both sides)."""
    import torch
    H0 = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    gx, gz, _ = iqcc.iqcc_dis_gradients(H0, th, ph, cap=n_gen)
    H0.close()
    taus = np.full(len(gx), tau)
    out = {"M0": len(c), "generators": f"top {len(gx)} DIS candidates of the loaded Hamiltonian, tau = {tau}"}
    for name, call in (("hash", lambda H: iqcc.iqcc_dress(H, gx, gz, taus)),
                       ("sorted_fuse1", lambda H: iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=1)),
                       (f"sorted_fuse{len(gx)}", lambda H: iqcc.iqcc_dress_sorted(H, gx, gz, taus, fuse=len(gx)))):
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=1 << 31)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        call(H)
        ev1.record(stream)
        ev1.synchronize()
        out[name] = {"ms": round(ev0.elapsed_time(ev1), 2), "M_after": len(H)}
        H.close()
    return out


def measure_plain_form(iqcc, n, x, z, c, th, ph, n_gen=8, tau=0.1, max_rows=120_000_000, budget_s=40.0):
    """The library's dress against the plain PyTorch-tensor form of the same
    step (baseline/plain_gpu.py: bitwise ops, torch.unique over key rows,
    index_add_) on the same GPU: the loaded Hamiltonian dressed by its top DIS
    candidates at tau, generator by generator while the table holds at most
    max_rows strings and the plain form stays within budget_s; wall time with a
    device synchronize on both sides of every call."""
    import torch
    from baseline.plain_gpu import PlainHamiltonian
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=1 << 31)
    gx, gz, _ = iqcc.iqcc_dis_gradients(H, th, ph, cap=n_gen)
    H.close()
    warm = PlainHamiltonian(n, x[:4096], z[:4096], c[:4096], device="cuda")  # first-call costs of the tensor ops
    warm.dress(gx[0], gz[0], tau)
    del warm
    P = PlainHamiltonian(n, x, z, c, device="cuda")
    m_in, t_plain = [], []
    for k in range(len(gx)):
        if len(P) > max_rows or sum(t_plain) > budget_s:
            break
        m_in.append(len(P))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P.dress(gx[k], gz[k], tau)
        torch.cuda.synchronize()
        t_plain.append(time.perf_counter() - t0)
    m_plain = len(P)
    del P
    torch.cuda.empty_cache()
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=1 << 31)
    t_lib = []
    for k in range(len(m_in)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        iqcc.iqcc_dress(H, gx[k:k + 1], gz[k:k + 1], np.array([tau]))
        torch.cuda.synchronize()
        t_lib.append(time.perf_counter() - t0)
    m_lib = len(H)
    H.close()
    terms = sum(m_in)
    return {"form": "plain PyTorch tensor ops on the same GPU (baseline/plain_gpu.py)",
            "generators": f"top {len(m_in)} DIS candidates of the loaded Hamiltonian, tau = {tau}",
            "M_in": m_in, "M_after": {"library": m_lib, "plain": m_plain},
            "ms_plain": [round(t * 1e3, 2) for t in t_plain], "ms_library": [round(t * 1e3, 2) for t in t_lib],
            "terms_per_s_plain": terms / sum(t_plain), "terms_per_s_library": terms / sum(t_lib),
            "speedup": round(sum(t_plain) / sum(t_lib), 2)}


def measure_partitioned(iqcc, n, x, z, c, th, ph, n_gen=8, tau=0.1):
    """The loaded Hamiltonian split in two contexts by the x bit of one qubit
    (App. B's bit-wise partitioning on one GPU, paper_2603_08883_gb300/
    partitioned.py), dressed by its top DIS candidates at tau; the qubit is
    the one most of those generators flip, and each generator that flips it
    dresses both parts through one set of pair bins (iqcc_dress_pair).  Then
    a term limit of half the terms over both parts (iqcc_prune_parts) against
    the same limit on one context.  Wall times with a device synchronize
    around each sequence."""
    import torch
    from paper_2603_08883_gb300 import partitioned as pt
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=1 << 31)
    gx, gz, _ = iqcc.iqcc_dis_gradients(H, th, ph, cap=n_gen)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    iqcc.iqcc_dress(H, gx, gz, np.full(len(gx), tau))
    torch.cuda.synchronize()
    t_one = time.perf_counter() - t0
    m_one = len(H)
    W = (n + 63) // 64
    flips = [sum((int(g[j // 64]) >> (j % 64)) & 1 for g in gx) for j in range(n)]
    qubit = int(np.argmax(flips))
    mx = np.zeros(W, np.uint64)
    mz = np.zeros(W, np.uint64)
    mx[qubit // 64] = np.uint64(1 << (qubit % 64))
    P = pt.PartitionedHamiltonian(n, x, z, c, mx, mz, capacity=1 << 31)
    parts_m0 = [len(h) for h in P.parts]
    crossing = sum(pt.generator_shift(a, b, mx, mz) != 0 for a, b in zip(gx, gz))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for a, b in zip(gx, gz):
        P.dress(a, b, tau)
    torch.cuda.synchronize()
    t_two = time.perf_counter() - t0
    m_two = len(P)
    limit = m_one // 2
    t0 = time.perf_counter()
    iqcc.iqcc_prune(H, 0.0, limit)
    torch.cuda.synchronize()
    t_cut_one = time.perf_counter() - t0
    t0 = time.perf_counter()
    P.prune(0.0, limit)
    torch.cuda.synchronize()
    t_cut_two = time.perf_counter() - t0
    out = {"split": f"x bit of qubit {qubit}", "parts_M0": parts_m0,
           "generators": f"top {len(gx)} DIS candidates of the loaded Hamiltonian, tau = {tau}",
           "crossing_generators": int(crossing), "M_after": {"one_context": m_one, "partitioned": m_two},
           "ms_one_context": round(t_one * 1e3, 2), "ms_partitioned": round(t_two * 1e3, 2),
           "term_limit": {"limit": limit, "ms_one_context": round(t_cut_one * 1e3, 2),
                          "ms_partitioned": round(t_cut_two * 1e3, 2), "M_after": [len(H), len(P)]}}
    H.close()
    P.close()
    return out


def measure_batch(iqcc, synth, n_problems=256, seed=1000, eps=1e-10, screens=20):
    """Many small Jordan-Wigner Hamiltonians (12..40 qubits, even, decay
    integrals, basis reference): one batched step against one single-problem
    iteration per problem, and repeated screening by graph replay."""
    import torch
    rng = np.random.Generator(np.random.PCG64(seed))
    probs, angles = [], []
    for b in range(n_problems):
        norb = int(rng.integers(6, 21))
        h, eri = synth.integrals("decay", norb, seed + b)
        n, x, z, c = synth.jordan_wigner(h, eri)
        probs.append((n, x.reshape(-1), z.reshape(-1), c))
        angles.append(synth.qmf_angles(n, "basis"))
    th = [a[0] for a in angles]
    ph = [a[1] for a in angles]
    out = {"problems": n_problems, "qubits": [int(p[0]) for p in probs], "terms": int(sum(len(p[3]) for p in probs)),
           "workload": "Jordan-Wigner of seeded decay integrals, 6-20 orbitals each, Hartree-Fock basis reference, "
                       "one generator per problem, eps 1e-10"}
    torch.cuda.synchronize()
    batch = iqcc.iqcc_batch_load(probs)
    iqcc.iqcc_batch_screen(batch, th, ph)  # tuning and capture
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(screens):
        iqcc.iqcc_batch_screen(batch, th, ph)
    out["screen_replay_ms"] = round((time.perf_counter() - t0) / screens * 1e3, 3)
    t0 = time.perf_counter()
    iqcc.iqcc_batch_step(batch, th, ph, eps)
    out["batched_step_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
    info = iqcc.iqcc_batch_get_info(batch)
    out["tuned_blocks"] = [info["blocks_energy"], info["blocks_group"], info["blocks_abc"]]
    batch.close()
    ctxs = [iqcc.iqcc_load_hamiltonian(p[0], p[1].reshape(-1, 1), p[2].reshape(-1, 1), p[3]) for p in probs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for H, t, p in zip(ctxs, th, ph):
        iqcc.iqcc_iterate(H, t, p, 1, eps, 0)
    torch.cuda.synchronize()
    out["one_context_per_problem_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
    for H in ctxs:
        H.close()
    return out


def profile_traffic(avg_rows):
    """DRAM bytes per dressed term of one dress (split + join) from the
    committed ncu summary (profiles/dress_pairs_jw100.md, line
    'dram_bytes_per_dressed_term:'), scaled to a dress of avg_rows rows; None
    when absent."""
    path = os.path.join(ROOT, "profiles", "dress_pairs_jw100.md")
    try:
        for line in open(path):
            if line.startswith("dram_bytes_per_dressed_term:"):
                return float(line.split(":")[1].split()[0]) * avg_rows
    except OSError:
        pass
    return None


# --------------------------------------------------------------------------- reference arm


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    from paper_2603_08883_gb300 import synth
    w = synth.WORKLOADS[args.workload]
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    rows = REFERENCE_ROWS
    for _ in range(args.warmup):
        oracle_dressed(w, n, x, z, c, th, ph, rows)
    tot, dt = 0, 0.0
    for _ in range(args.steps):
        d, t = oracle_dressed(w, n, x, z, c, th, ph, rows)
        tot += d
        dt += t
    value = tot / dt
    sample = (f"each step: one oracle iteration (DIS, {w.n_gen} x (A,B,C + dress + term limit), compression, "
              f"energy) on the first {rows} of the {len(c)} strings of the {w.n_qubits}-qubit Hamiltonian")
    print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
                      "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
                      "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                      "impl": "reference",
                      "config": workload_config(w, {"sample_rows": rows}),
                      "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
                      "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}),
          flush=True)


# --------------------------------------------------------------------------- GPU arm


def run_gpu(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2603_08883_gb300 import iqcc, synth

    w = synth.WORKLOADS[args.workload]
    if args.max_terms > 0:
        import dataclasses
        w = dataclasses.replace(w, max_terms=args.max_terms, capacity=2 * args.max_terms,
                                notes=w.notes + f" (profiling case: term limit lowered to {args.max_terms})")
    if world > 1:
        w = workload_for_rank(w, rank)
    n, x, z, c = synth.workload_hamiltonian(w)
    th, ph = synth.workload_angles(w)
    M0 = len(c)
    log(f"generated {w.name}: n={n} M0={M0}")
    stream = torch.cuda.current_stream()
    capacity = w.capacity

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # ---------------- device-resident run
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=capacity)
    log(f"loaded: M={len(H)}")
    for it in range(args.warmup):
        r = iqcc.iqcc_iterate(H, th, ph, w.n_gen, w.eps, w.max_terms)
        free_b, total_b = torch.cuda.mem_get_info()
        log(f"warmup {it}: M {r['M_before']} -> peak {r['M_peak']} -> {r['M']}, E={r['energy']:.9f}, "
            f"device free {free_b / 2**30:.1f} GiB")
    M_start = len(H)
    flush = M_start * (16 * ((n + 63) // 64) + 8) < 2 * L2_BYTES
    scratch = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda") if flush else None
    iqcc.iqcc_reset_stats(H)
    recs = []
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            if scratch is not None:
                scratch.zero_()
            recs.append(iqcc.iqcc_iterate(H, th, ph, w.n_gen, w.eps, w.max_terms))
        ev1.record(stream)
        barrier()
        wall = time.perf_counter() - t0
    dev_s = ev0.elapsed_time(ev1) / 1e3
    log(f"timed: {args.steps} iterations in {dev_s:.3f} s; M {[r['M'] for r in recs]}")
    stats = iqcc.iqcc_get_stats(H)
    dressed = sum(r["dressed_terms"] for r in recs)
    t_max, total_dressed = reduce_over_ranks(dist, dev_s, dressed, "cuda")

    # ---------------- adjoint pass (dE/dtheta, dE/dphi, dE/dtau) on the capped H, after the timed region
    adjoint = sort_variant = screening = plain_form = partitioned = None
    if rank == 0 and not args.no_extras:
        adjoint = measure_adjoint(iqcc, H, n, th, ph, stream)
        adjoint["joint_optimisation"] = measure_joint_optimisation(iqcc, H, th, ph)
        screening = measure_screening(iqcc, H, th, ph)

    # ---------------- end to end through host buffers (pinned), N = 1 path of a user
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        hx, hz, hc = iqcc.iqcc_export(H)
        W = hx.shape[1]
        cap_rows = max(w.max_terms if w.max_terms > 0 else 0, len(hc)) + 1

        def pinned(shape, dtype):
            nbytes = int(np.prod(shape)) * np.dtype(dtype).itemsize
            t = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
            return t.numpy().view(dtype).reshape(shape)

        bufs = [(pinned((cap_rows, W), np.uint64), pinned((cap_rows, W), np.uint64), pinned((cap_rows,), np.float64))
                for _ in range(2)]
        m = len(hc)
        bufs[0][0][:m], bufs[0][1][:m], bufs[0][2][:m] = hx, hz, hc
        del hx, hz, hc
        H.close()
        h2d = d2h = 0
        e_dressed = 0
        phases = {"load_s": 0.0, "iterate_s": 0.0, "export_s": 0.0}
        barrier()
        t0 = time.perf_counter()
        for k in range(args.e2e_steps):
            src, dst = bufs[k % 2], bufs[(k + 1) % 2]
            ta = time.perf_counter()
            Hk = iqcc.iqcc_load_hamiltonian(n, src[0][:m], src[1][:m], src[2][:m], capacity=capacity)
            torch.cuda.synchronize()
            tb = time.perf_counter()
            r = iqcc.iqcc_iterate(Hk, th, ph, w.n_gen, w.eps, w.max_terms)
            torch.cuda.synchronize()
            tc = time.perf_counter()
            ox, oz, oc = iqcc.iqcc_export_rows(Hk, out=dst)
            phases["load_s"] += tb - ta
            phases["iterate_s"] += tc - tb
            phases["export_s"] += time.perf_counter() - tc
            h2d += m * (2 * W * 8 + 8) + 2 * n * 8
            d2h += len(oc) * (2 * W * 8 + 8) + 8
            m = len(oc)
            e_dressed += r["dressed_terms"]
            Hk.close()
            log(f"e2e step {k}: M -> {m}")
        barrier()
        e_wall = time.perf_counter() - t0
        e2e = {"value": e_dressed / e_wall, "unit": UNIT, "h2d_bytes_per_step": h2d // args.e2e_steps,
               "d2h_bytes_per_step": d2h // args.e2e_steps, "steps": args.e2e_steps,
               "phases_s_per_step": {k: round(v / args.e2e_steps, 4) for k, v in phases.items()},
               "path": "per step: iqcc_load_hamiltonian from pinned host arrays, iqcc_iterate, iqcc_export_rows "
                       "(storage order, no sort) to pinned host arrays, the next step's input; wall clock"}
    else:
        H.close()
    batch_variant = None
    if rank == 0 and not args.no_extras:  # after the capped Hamiltonian is released
        sort_variant = measure_sort_variant(iqcc, n, x, z, c, th, ph, stream)
        plain_form = measure_plain_form(iqcc, n, x, z, c, th, ph)
        partitioned = measure_partitioned(iqcc, n, x, z, c, th, ph)
        batch_variant = measure_batch(iqcc, synth)

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    # ---------------- roofline of the dress (split + join of one generator)
    peak, peak_kind = measured_peak()
    n_dress = max(stats["n_dress"], 1)
    dress_s = stats["dress_kernel_ms"] / 1e3
    achieved = stats["dress_bytes"] / dress_s / 1e9 if dress_s > 0 else 0.0
    avg_rows = stats["dressed_terms"] / n_dress
    # bytes the pair-partition dress itself moves: the split reads and writes
    # every live row (commuting rows to the other buffer, anticommuting rows to
    # their bins); the join reads the bins and writes the rotated rows and the
    # appended partners
    row_b = 16 * (1 if n <= 64 else 2 if n <= 128 else 4) + 8
    moved = row_b * (2 * stats["dressed_terms"] + 2 * stats["anticommuting"] + stats["appended"])
    shares = {"dress": stats["dress_kernel_ms"], "key_index": stats["hash_ms"],
              "compression": stats["prune_ms"], "dis_screening": stats["dis_ms"],
              "energy_abc": stats["energy_kernel_ms"]}
    tot_ms = sum(shares.values())
    roofline = {"bound": "hbm", "kernel": "dress of one generator: k_pair_split + k_pair_join (bin and tile "
                                          "counts from the preceding A,B,C pass)",
                "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                "traffic": profile_traffic(avg_rows),
                "bytes_per_launch": stats["dress_bytes"] / n_dress, "launches": stats["n_dress"],
                "avg_launch_ms": stats["dress_kernel_ms"] / n_dress,
                "bytes_model": "16W M_in + 16 M_anti + (16W+8) M_new per dress (the method's own bytes)",
                "moved_bytes_per_launch": moved / n_dress,
                "moved_frac": round(moved / dress_s / 1e9 / peak, 4) if dress_s > 0 else None,
                "moved_model": "(16W+8)(2 M_in + 2 M_anti + M_new): split copies every row once, "
                               "join reads the bins and writes rotated and appended rows",
                "anticommuting_per_launch": stats["anticommuting"] / n_dress,
                "appended_per_launch": stats["appended"] / n_dress,
                "device_ms_share": {k: round(v / tot_ms, 4) for k, v in shares.items()} if tot_ms else {},
                "adjoint_pass": adjoint, "sort_variant": sort_variant, "batch_variant": batch_variant,
                "learned_screening": screening, "plain_gpu_form": plain_form, "partitioned_variant": partitioned}

    # ---------------- oracle on the host cores (N = 1 only)
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        rows = REFERENCE_ROWS
        d, t = oracle_dressed(w, n, x, z, c, th, ph, rows)
        cpu = {"value": d / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"one oracle iteration (DIS, {w.n_gen} x (A,B,C + dress + term limit), compression, "
                         f"energy) on the first {rows} of the {M0} strings; {d} dressed terms in {t:.2f} s"}

    line = {"metric": METRIC, "value": total_dressed / t_max, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(w, {
                "M0": M0, "M_first_timed": M_start, "M_last": recs[-1]["M"] if recs else M_start,
                "iterations": f"{args.warmup + 1}..{args.warmup + args.steps}",
                "s_per_iteration": t_max / args.steps,
                "l2": ("flushed before each step (256 MiB write)" if flush else
                       f"inputs larger than L2: H >= {M_start * (16 * ((n + 63) // 64) + 8) / 2**20:.0f} MiB "
                       "at the first timed step"),
                "energies": [r["energy"] for r in recs],
                "wall_s": wall}),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": stats["kernel_launches"], "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def log(msg):
    if int(os.environ.get("RANK", "0")) == 0:
        sys.stderr.write(f"[bench {time.strftime('%H:%M:%S')}] {msg}\n")
        sys.stderr.flush()


def main():
    faulthandler.enable()
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
