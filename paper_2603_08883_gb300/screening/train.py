"""Train the term-screening perceptron on untruncated iQCC runs, and compare
the learned term limit with the magnitude limit on held-out problems.

    python -m paper_2603_08883_gb300.screening.train --out paper_2603_08883_gb300/screening/model_jw.npz
    python -m paper_2603_08883_gb300.screening.train --evaluate paper_2603_08883_gb300/screening/model_jw.npz
    python -m paper_2603_08883_gb300.screening.train --evaluate-large paper_2603_08883_gb300/screening/model_jw.npz \
        --qubits 124 --budget 1e8 --ref-budget 8e8

Data: Jordan-Wigner Hamiltonians of seeded decay integrals (12-16 orbitals,
24-32 qubits) and d-block integrals (16-20 orbitals, 32-40 qubits),
Hartree-Fock basis reference, iterations of 4 generators with eps = 1e-10 and
no term limit.  Each problem is run once to record its
generators and amplitudes, then replayed with those generators forced; before
every iteration the features of every term (G = that iteration's generators)
and the target log10 |C_T E_fut(T)| are taken, E_fut over the generators of
that iteration and the next (at most 8): the exact energy change, after those
generators, of removing T now (floored at 1e-20).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def problem(norb: int, seed: int, kind: str = "decay"):
    from .. import synth
    h, eri = synth.integrals(kind, norb, seed)
    n, x, z, c = synth.jordan_wigner(h, eri)
    th, ph = synth.qmf_angles(n, "basis")
    return n, x, z, c, th, ph


def samples(norb: int, seed: int, iters: int, per_iter: int, rng, kind: str = "decay"):
    from .. import iqcc
    n, x, z, c, th, ph = problem(norb, seed, kind)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    rec = []
    for _ in range(iters):
        try:
            rec.append(iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 0))
        except iqcc.IqccError as e:  # the untruncated run outgrew the device: keep the iterations done
            if e.status not in (3, 4):  # IQCC_ERR_OOM, IQCC_ERR_CAPACITY
                raise
            break
    H.close()
    iters = len(rec)
    H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
    X, Y = [], []
    for it in range(iters):
        r = rec[it]
        nxt = rec[it + 1] if it + 1 < iters else None
        gx = r["gx"] if nxt is None else np.concatenate([r["gx"], nxt["gx"]])[:8]
        gz = r["gz"] if nxt is None else np.concatenate([r["gz"], nxt["gz"]])[:8]
        tau = r["tau"] if nxt is None else np.concatenate([r["tau"], nxt["tau"]])[:8]
        f = iqcc.iqcc_term_features(H, th, ph, r["gx"], r["gz"])
        fut = iqcc.iqcc_future_energies(H, th, ph, gx, gz, tau)
        c_now = iqcc.iqcc_export(H)[2]
        y = np.log10(np.abs(c_now * fut) + 1e-20)  # terms with no effect sit at the floor
        pick = rng.choice(len(y), size=min(per_iter, len(y)), replace=False)
        X.append(f[pick])
        Y.append(y[pick].astype(np.float32))
        iqcc.iqcc_iterate(H, th, ph, 0, 1e-10, 0, forced_x=r["gx"], forced_z=r["gz"], forced_tau=r["tau"])
    H.close()
    return np.concatenate(X), np.concatenate(Y)


def fit(X, Y, epochs: int, seed: int):
    import torch
    torch.manual_seed(seed)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    net = torch.nn.Sequential(torch.nn.Linear(8, 256), torch.nn.ReLU(), torch.nn.Linear(256, 256), torch.nn.ReLU(),
                              torch.nn.Linear(256, 1)).to(dev)
    Xt = torch.from_numpy(X).to(dev)
    Yt = torch.from_numpy(Y).to(dev)
    opt = torch.optim.Adam(net.parameters(), lr=1e-3)
    sched = torch.optim.lr_scheduler.StepLR(opt, step_size=max(1, epochs // 3), gamma=0.3)
    n = len(Xt)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, device=dev)
        tot = 0.0
        for i in range(0, n, 4096):
            idx = perm[i:i + 4096]
            loss = torch.mean((net(Xt[idx]).squeeze(1) - Yt[idx]) ** 2)
            opt.zero_grad()
            loss.backward()
            opt.step()
            tot += float(loss.detach()) * len(idx)
        sched.step()
        losses.append(tot / n)
    l1, l2, l3 = net[0], net[2], net[4]
    cpu = lambda t: t.detach().cpu().numpy().astype(np.float32)
    return {"w1": cpu(l1.weight), "b1": cpu(l1.bias), "w2": cpu(l2.weight), "b2": cpu(l2.bias),
            "w3": cpu(l3.weight).reshape(-1), "b3": np.float32(float(l3.bias))}, losses


def evaluate(model_path: str, norbs=(12, 13, 14, 15), seeds=(4100, 4101, 4102, 4103), iters: int = 5,
             budget: float = 0.3, floors=(0.0, 0.5)):
    """|E - E_untruncated| after `iters` iterations with a term limit of
    budget x the untruncated run's final size: magnitude, and learned with
    each magnitude floor."""
    from .. import iqcc
    from . import load_model
    model = load_model(model_path)
    out = []
    for norb, seed in zip(norbs, seeds):
        n, x, z, c, th, ph = problem(norb, seed)
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
        for _ in range(iters):
            r = iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, 0)
        e_ref, m_ref = r["energy"], r["M"]
        H.close()
        cap = max(1000, int(budget * m_ref))
        res = {"qubits": n, "seed": seed, "untruncated_terms": m_ref, "term_limit": cap, "E_untruncated": e_ref}
        for name, mode, floor in [("magnitude", 0, 0.0)] + [(f"learned_floor{f:g}", 1, f) for f in floors]:
            H = iqcc.iqcc_load_hamiltonian(n, x, z, c)
            iqcc.iqcc_set_screening_model(H, *model)
            iqcc.iqcc_set_screening_floor(H, floor)
            for _ in range(iters):
                r = iqcc.iqcc_iterate(H, th, ph, 4, 1e-10, cap, screening=mode)
            res["error_" + name] = abs(r["energy"] - e_ref)
            H.close()
        out.append(res)
    return out


def evaluate_large(model_path: str, qubits: int = 124, seed: int = 124, iters: int = 6, n_gen: int = 8,
                   eps: float = 1e-8, budget: int = 100_000_000, ref_budget: int = 800_000_000,
                   floors=(0.0, 0.5)):
    """The learned term limit beyond the training sizes: Jordan-Wigner
    Hamiltonian of seeded d-block integrals (as the 100-qubit workload, with
    qubits / 2 orbitals), Hartree-Fock basis reference, `iters` iterations of
    `n_gen` DIS generators, prune eps.  Runs with the term limit `budget`
    (magnitude, then learned with each magnitude floor) against the same run
    with the limit `ref_budget` standing in for the untruncated one (which
    does not fit at this size); energies after every iteration."""
    from .. import iqcc, synth
    from . import load_model
    t0 = time.time()
    h, eri = synth.integrals("dblock", qubits // 2, seed)
    n, x, z, c = synth.jordan_wigner(h, eri)
    th, ph = synth.qmf_angles(n, "basis", seed)
    out = {"qubits": n, "seed": seed, "M0": len(c), "iterations": iters, "generators": n_gen, "eps": eps,
           "term_limit": budget, "reference_term_limit": ref_budget,
           "generate_s": round(time.time() - t0, 1)}
    model = load_model(model_path)
    runs = [("reference", ref_budget, 0, 0.0), ("magnitude", budget, 0, 0.0)]
    runs += [(f"learned_floor{f:g}", budget, 1, f) for f in floors]
    for name, cap, mode, floor in runs:
        t0 = time.time()
        H = iqcc.iqcc_load_hamiltonian(n, x, z, c, capacity=2 * cap)
        if mode:
            iqcc.iqcc_set_screening_model(H, *model)
            iqcc.iqcc_set_screening_floor(H, floor)
        energies, sizes = [], []
        for _ in range(iters):
            r = iqcc.iqcc_iterate(H, th, ph, n_gen, eps, cap, screening=mode)
            energies.append(r["energy"])
            sizes.append(r["M"])
        H.close()
        out[name] = {"energies": energies, "M": sizes, "seconds": round(time.time() - t0, 1)}
    ref = out["reference"]["energies"]
    for name, _, _, _ in runs[1:]:
        out[name]["error_vs_reference"] = [abs(a - b) for a, b in zip(out[name]["energies"], ref)]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None)
    ap.add_argument("--evaluate", default=None)
    ap.add_argument("--epochs", type=int, default=12)
    ap.add_argument("--iters", type=int, default=5)
    ap.add_argument("--per-iter", type=int, default=60000)
    ap.add_argument("--evaluate-large", default=None)
    ap.add_argument("--qubits", type=int, default=124)
    ap.add_argument("--budget", type=float, default=1e8)
    ap.add_argument("--ref-budget", type=float, default=8e8)
    args = ap.parse_args()
    if args.out:
        rng = np.random.Generator(np.random.PCG64(0))
        t0 = time.time()
        X, Y = [], []
        for norb, seed, kind, iters in [(12, 3000, "decay", args.iters), (12, 3001, "decay", args.iters),
                                        (13, 3002, "decay", args.iters), (14, 3003, "decay", args.iters),
                                        (15, 3004, "decay", args.iters), (16, 3005, "decay", args.iters),
                                        (16, 3006, "dblock", 4), (18, 3007, "dblock", 3), (20, 3008, "dblock", 3)]:
            xs, ys = samples(norb, seed, iters, args.per_iter, rng, kind)
            X.append(xs)
            Y.append(ys)
        X, Y = np.concatenate(X), np.concatenate(Y)
        w, losses = fit(X, Y, args.epochs, 0)
        np.savez(args.out, **w, samples=len(X), losses=np.array(losses), target_var=float(np.var(Y)))
        print(json.dumps({"samples": len(X), "target_var": float(np.var(Y)), "losses": losses,
                          "seconds": time.time() - t0}))
    if args.evaluate:
        print(json.dumps(evaluate(args.evaluate)))
    if args.evaluate_large:
        print(json.dumps(evaluate_large(args.evaluate_large, qubits=args.qubits, seed=args.qubits,
                                        budget=int(args.budget), ref_budget=int(args.ref_budget))))


if __name__ == "__main__":
    main()
