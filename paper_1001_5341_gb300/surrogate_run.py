"""Train and evaluate the learned near-field surrogate on FDTD runs.

    python -m paper_1001_5341_gb300.surrogate_run [--train-runs N] [--test-runs M] [--steps S] [--out report.json]

1. Data: seeded Gaisser-Hillas showers on the 128x128x512 CPML grid
   (workloads.surrogate_grid / surrogate_runs), 2048 FDTD steps per run, 64
   antennas per run (all of them from one run, Sec. III.B); training and
   held-out showers come from different seeds.
2. Two networks (different seeds) trained by the library's kernels.
3. Accuracy on the held-out showers: relative L2 of the 1024-sample trace
   (every second step) against FDTD.
4. Fallback gate: the two networks' disagreement; for each target error the
   gate threshold is calibrated on half of the held-out antennas and applied
   to the other half: accepted antennas use the surrogate, the rest FDTD.
5. Throughput: surrogate pulses/s at batch 4096 (one network; CUDA events)
   against FDTD pulses/s (antennas per run / run time), and the effective
   pulses/s with the fallback.
Prints one JSON report (and writes it with --out).
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--train-runs", type=int, default=200)
    ap.add_argument("--test-runs", type=int, default=24)
    ap.add_argument("--probes", type=int, default=64)
    ap.add_argument("--steps", type=int, default=12000, help="optimiser steps per network")
    ap.add_argument("--batch", type=int, default=32)
    ap.add_argument("--hidden", type=int, default=512)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--zs", type=float, default=10.5, help="axial-offset feature scale (metres)")
    ap.add_argument("--out", default="")
    args = ap.parse_args(argv)

    import torch
    torch.cuda.set_device(0)
    import workloads as W
    from paper_1001_5341_gb300 import surrogate as S

    log = lambda m: print(m, file=sys.stderr, flush=True)
    grid = W.surrogate_grid()
    decim = 1
    train = S.generate(grid, W.surrogate_runs(seed=5000, n_runs=args.train_runs, n_probes=args.probes), decim, log)
    test = S.generate(grid, W.surrogate_runs(seed=9000, n_runs=args.test_runs, n_probes=args.probes), decim, log)
    geo = S.Geometry.of(grid, decim=decim, m=8, feat=(0.6, 0.3, 0.0, args.zs))
    fdtd_run_s = (train.fdtd_s + test.fdtd_s) / (args.train_runs + args.test_runs)
    fdtd_pps = args.probes / fdtd_run_s

    tr = train.trace.double().cpu().numpy()
    s = np.abs(train.q.double().cpu().numpy()).max(axis=1)
    c_out = float(np.sqrt(np.mean((tr / s[:, None]) ** 2)))
    ntr = tr.shape[0]
    nets = []
    t_train = 0.0
    for seed in (1, 2):
        net = S.Net(geo, hidden=args.hidden, seed=seed, c_out=c_out)
        rng = np.random.default_rng(seed)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for it in range(args.steps):
            idx = torch.tensor(rng.choice(ntr, size=args.batch, replace=False), device="cuda")
            lr = args.lr if it < 0.7 * args.steps else args.lr * 0.2
            loss = net.train_batch(train.q[idx].contiguous(), train.rz[idx].contiguous(),
                                   train.trace[idx].contiguous(), lr)
            if it % 2000 == 0:
                log(f"net {seed} step {it} loss {float(loss.item()):.4e}")
        torch.cuda.synchronize()
        t_train += time.perf_counter() - t0
        nets.append(net)

    # accuracy on held-out showers, 1024-sample traces (every second step)
    ref = test.trace.double().cpu().numpy()[:, 1::2]
    preds = [n.predict(test.q, test.rz).double().cpu().numpy()[:, 1::2] for n in nets]
    err = S.rel_l2(preds[0], ref)
    mean_pred = 0.5 * (preds[0] + preds[1])
    gate = np.linalg.norm(preds[0] - preds[1], axis=1) / np.maximum(np.linalg.norm(mean_pred, axis=1), 1e-300)
    rng = np.random.default_rng(0)
    perm = rng.permutation(len(err))
    cal, ev = perm[: len(err) // 2], perm[len(err) // 2:]

    # surrogate throughput, batch 4096 (one network)
    nb = 4096
    qb = test.q[torch.arange(nb, device="cuda") % test.q.shape[0]].contiguous()
    rb = test.rz[torch.arange(nb, device="cuda") % test.rz.shape[0]].contiguous()
    nets[0].predict(qb, rb)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    reps = 3
    for _ in range(reps):
        nets[0].predict(qb, rb)
    e1.record()
    torch.cuda.synchronize()
    sur_pps = reps * nb / (e0.elapsed_time(e1) * 1e-3)

    gates = {}
    for target in (0.01, 0.05, 0.10, 0.20):
        # largest threshold whose accepted calibration antennas meet the target at the 90th percentile
        order = np.argsort(gate[cal])
        thr = -1.0
        for m in range(1, len(order) + 1):
            acc = cal[order[:m]]
            if np.percentile(err[acc], 90) <= target:
                thr = gate[cal[order[m - 1]]]
        accepted = ev[gate[ev] <= thr] if thr >= 0 else ev[:0]
        frac = len(accepted) / len(ev)
        eff = 1.0 / (frac / sur_pps + (1 - frac) / fdtd_pps)
        gates[f"{target:g}"] = {
            "accepted_fraction": round(frac, 4),
            "accepted_err_p50": float(np.median(err[accepted])) if len(accepted) else None,
            "accepted_err_p90": float(np.percentile(err[accepted], 90)) if len(accepted) else None,
            "effective_pulses_per_s": round(eff, 1), "effective_vs_fdtd": round(eff / fdtd_pps, 2)}

    rep = {
        "what": "learned surrogate (learned bin response in retarded time, summed over the profile) vs FDTD",
        "grid": grid.describe(), "train_showers": args.train_runs, "test_showers": args.test_runs,
        "antennas_per_run": args.probes, "trace_samples": ref.shape[1], "params_per_net": nets[0].n_params,
        "hidden": args.hidden, "optimizer_steps": args.steps, "batch": args.batch, "feature_zs": args.zs,
        "train_seconds_two_nets": round(t_train, 1),
        "fdtd_seconds_per_run": round(fdtd_run_s, 4), "fdtd_pulses_per_s": round(fdtd_pps, 1),
        "surrogate_pulses_per_s_batch4096": round(sur_pps, 1), "surrogate_vs_fdtd": round(sur_pps / fdtd_pps, 1),
        "test_rel_l2": {"p10": float(np.percentile(err, 10)), "p50": float(np.median(err)),
                        "p90": float(np.percentile(err, 90)), "frac_le_1pct": float(np.mean(err <= 0.01)),
                        "frac_le_10pct": float(np.mean(err <= 0.10))},
        "fallback_gate": gates,
    }
    print(json.dumps(rep), flush=True)
    if args.out:
        with open(args.out, "w") as f:
            json.dump(rep, f, indent=1)


if __name__ == "__main__":
    main()
