#!/usr/bin/env python3
"""Throughput of the 3D Yee FDTD near-field path on GB300.

One bench "step" is one leapfrog step of the whole hot path over the grid:
H-curl update, E-curl update with the moving shower's current, CPML, detector
readout.  The workload is the 384 x 384 x 1536-cell ice grid (dx = 2 cm,
10-cell CPML, Greisen shower of seeded energy, NKG lateral spread, 64
detectors at r = 1-5 m).  Metric: Gcell-updates/s = cells x steps / time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank runs an independent replica (its own seeded
shower) on its own GPU; there is no data-path communication.  Rank 0 prints
one JSON line.  ``--impl reference`` times the FP64 CPU oracle instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import workloads as W  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")
FALLBACK_HBM_GBS = 6800.0


def bytes_per_cell(w) -> float:
    """Compulsory HBM bytes per cell-update: six float32 components read and
    written once (48 B), plus the CPML memory (4 psi per slab cell per axis,
    each read and written, 8 B) averaged over the grid."""
    b = 48.0
    if w.boundary == W.CPML:
        P = w.npml
        W_ = 2 * P + 1
        slab = (W_ * w.ny * w.nz + w.nx * W_ * w.nz + w.nx * w.ny * W_)
        b += 4 * 8.0 * slab / w.cells
    return b


def field_gb(w) -> float:
    """Device bytes of the two field sets: 2 x 6 float32 arrays over the
    node grid with x rows padded to 32 floats."""
    pitch = (w.nx + 1 + 31) // 32 * 32
    return 2 * 6 * (w.nz + 1) * (w.ny + 1) * pitch * 4 / 1e9


def hbm_peak():
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_source_hash(files):
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1001_5341_gb300", "csrc")
    for fn in files:
        with open(os.path.join(csrc, fn), "rb") as f:
            h.update(fn.encode() + f.read())
    return h.hexdigest()[:16]


def ncu_record(kernel_name, workload_name):
    """The committed ncu DRAM capture of this kernel on this workload, or None
    when none exists or a source file it lists changed since."""
    try:
        with open(TRAFFIC) as f:
            data = json.load(f)
    except Exception:
        return None
    # one record per (kernel, workload): "<kernel>@<workload>", or the kernel's own name
    rec = data.get(f"{kernel_name}@{workload_name}") or data.get(kernel_name)
    if not rec or rec.get("workload") != workload_name:
        return None
    if rec.get("source_hash") != kernel_source_hash(rec.get("sources", [])):
        return None
    return rec


def ncu_traffic(kernel_name, workload_name):
    """DRAM bytes per cell-update of the 3D step kernel (see ncu_record)."""
    rec = ncu_record(kernel_name, workload_name)
    return rec.get("dram_bytes_per_cell") if rec else None


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(vals, ws, device="cpu"):
    """Element-wise maximum of a list of floats over the ranks of the process
    group (the slowest replica sets the time); the identity with one rank."""
    import torch
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    if ws > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.cpu()]


WORKLOAD_SEEDS = {"greisen384": 2002, "gh640": 3003}


def replica_workload(rank, workload="greisen384", **kw):
    """The benchmark shower of one replica: rank r draws the workload's seed + r
    (greisen384: 384 x 384 x 1536, Greisen shower; gh640: 640 x 640 x 2048,
    dx = 3 cm, 3-6 Gaisser-Hillas subshowers over 40 m, 256 detectors)."""
    make = {"greisen384": W.greisen384, "gh640": W.gh640}[workload]
    return make(seed=WORKLOAD_SEEDS[workload] + rank, **kw)


def near_field_vs_fraunhofer(fd, sim, w, stream):
    """The detectors' theta-hat spectra (fdtd_trace_spectrum over the whole
    trace; the CPML leaves no reflections) against the far-field formula
    eq. 1d_appro for the same charge table, in a frame centred on the
    charge-weighted middle of the shower:
        E_theta = -i w mu0/(4 pi) sin(theta) exp(ikR)/R sum q(z') dz' exp(i p z'),
        p = w (1/v - n cos(theta)/c).
    Reports, per frequency, the median and spread of |E| / |E_formula| and
    the median far-field parameter l^2 sin^2(theta) / (lambda R), l the
    charge-weighted rms length of the shower."""
    import torch
    q, _ = fd.tables(w)
    zq = w.z0 + w.bin_dz * np.arange(q.size)
    aq = np.abs(q)
    zc = float((zq * aq).sum() / aq.sum())
    l_rms = float(np.sqrt(((zq - zc) ** 2 * aq).sum() / aq.sum()))
    ax, ay = (w.nx // 2) * w.dx, (w.ny // 2) * w.dx
    node = np.floor(w.probes_xyz / w.dx + 0.5) * w.dx
    r = np.hypot(node[:, 0] - ax, node[:, 1] - ay)
    R = np.hypot(r, node[:, 2] - zc)
    th = np.arctan2(r, node[:, 2] - zc)
    freqs = np.array([50e6, 100e6, 150e6, 200e6, 300e6])
    tr = torch.empty((w.probes_xyz.shape[0], sim.max_steps, 2), dtype=torch.float32, device="cuda")
    sim.probes(out=tr)
    E = np.abs(fd.trace_spectrum(tr, w.dt, freqs, t0=w.dt, coef=fd.theta_coef(th), stream=stream).cpu().numpy())
    n_idx = math.sqrt(w.eps_r)
    mu0 = 4e-7 * math.pi
    om = 2 * math.pi * freqs
    ratio = np.zeros_like(E)
    for p in range(E.shape[0]):
        pz = om[:, None] * (1.0 / w.v - n_idx * math.cos(th[p]) / W.C0)
        I = np.abs(((q * w.bin_dz)[None, :] * np.exp(1j * pz * (zq - zc)[None, :])).sum(axis=1))
        Ef = om * mu0 / (4 * math.pi) * math.sin(th[p]) / R[p] * I
        ratio[p] = E[p] / Ef
    lam = W.C0 / (n_idx * freqs)
    ff = np.median(l_rms ** 2 * np.sin(th)[:, None] ** 2 / (lam[None, :] * R[:, None]), axis=0)
    return {"frame": f"charge-weighted middle z = {zc:.2f} m, rms length {l_rms:.2f} m",
            "detectors": int(E.shape[0]), "R_m": [round(float(R.min()), 1), round(float(R.max()), 1)],
            "freqs_MHz": (freqs / 1e6).tolist(),
            "median_E_over_formula": np.round(np.median(ratio, axis=0), 3).tolist(),
            "p10_E_over_formula": np.round(np.percentile(ratio, 10, axis=0), 3).tolist(),
            "p90_E_over_formula": np.round(np.percentile(ratio, 90, axis=0), 3).tolist(),
            "within_10pct": np.round(np.mean(np.abs(ratio - 1) <= 0.1, axis=0), 3).tolist(),
            "median_l2sin2_over_lambdaR": np.round(ff, 2).tolist()}


def run_ours(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1001_5341_gb300 as fd

    # each replica draws its own shower; rank 0 runs the named seed
    w = replica_workload(rank, args.workload, steps=args.warmup + args.steps, **({"nz": args.nz} if args.nz else {}))
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = fd.Simulation.from_workload(w, max_steps=args.warmup + args.steps, stream=stream,
                                          kernel=args.kernel if args.kernel >= 0 else None)
        sim.step(args.warmup)
        sim.sync()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        l0 = sim.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        sim.timing_begin(4 * args.steps)
        ev0.record(stream)
        sim.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        kern_ms, kern_launches = sim.timing_end()
        launches = sim.launches - l0
        ms = ev0.elapsed_time(ev1)
        clk = clocks.stop()
        try:
            sim.energy()   # stability check after the timed region
            stable = True
        except fd.FdtdError:
            stable = False

        near = None
        if w.profile["kind"] == "gh" and rank == 0 and args.warmup + args.steps >= w.steps:
            near = near_field_vs_fraunhofer(fd, sim, w, stream)

        # end to end through the public API with host buffers: upload the
        # shower and detector tables, step, read the traces back to the host
        q, lw = fd.tables(w)
        xyz = np.ascontiguousarray(w.probes_xyz)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.reset()
        sim.set_shower(q, w.z0, w.bin_dz, w.v, lw, w.lateral["L"])
        sim.set_probes(xyz, args.steps)
        sim.step(args.steps)
        tr = sim.probes()
        t1 = time.perf_counter()
        e2e_s = t1 - t0
        h2d = q.nbytes + lw.nbytes + xyz.nbytes
        d2h = tr.nbytes
        kernel_name = sim.kernel_name
        sim.close()

    ms_max, e2e_ms_max = max_over_ranks([ms, e2e_s * 1e3], ws, device="cuda")
    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return None

    cells = w.cells
    value = ws * cells * args.steps / (ms_max * 1e-3) / 1e9
    b = bytes_per_cell(w)
    peak, peak_kind = hbm_peak()
    # a launch of either path reads the fields and the CPML memory once and
    # writes them once: b bytes per cell and launch (the two-step path's launch
    # advances two steps)
    achieved = b * cells * kern_launches / (kern_ms * 1e-3) / 1e9 if kern_ms > 0 else None
    steps_per_launch = round(args.steps / kern_launches) if kern_launches else None
    traffic = ncu_traffic(kernel_name, w.name)
    line = {
        "metric": "Gcell-updates/s", "value": round(value, 3), "unit": "Gcell/s",
        "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**w.describe(), "seed": WORKLOAD_SEEDS[args.workload], "inputs_vs_l2": f"fields {field_gb(w):.1f} GB >> 129 MB L2 (no L2 flush needed)",
                   "parallelism": f"replicas{ws}" if ws > 1 else "single-gpu",
                   "replica_seeds": f"{WORKLOAD_SEEDS[args.workload]} + rank"},
        "roofline": {"bound": "hbm", "kernel": kernel_name,
                     "achieved": round(achieved, 1) if achieved else None,
                     "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": round(achieved / peak, 4) if achieved else None,
                     "frac_of_nominal_7900": round(achieved / 7900.0, 4) if achieved else None,
                     "bytes_per_cell_alg": round(b, 3),
                     "traffic": (traffic * cells if traffic else None),
                     "steps_per_launch": steps_per_launch,
                     # Gcell-updates/s x bytes per cell-update of a one-step
                     # pass, against the same peak (above 1 only by blocking)
                     "cell_update_equivalent_frac": round(value * b / peak, 4),
                     "kernel_ms_per_step": round(kern_ms / args.steps, 5),
                     "kernel_launches_timed": kern_launches},
        "e2e": {"value": round(ws * cells * args.steps / (e2e_ms_max * 1e-3) / 1e9, 3),
                "unit": "Gcell/s", "h2d_bytes_per_step": round(h2d / args.steps, 1),
                "d2h_bytes_per_step": round(d2h / args.steps, 1),
                "what": "reset + set_shower + set_probes (host tables) + step(K) + probes() to host"},
        "gpu_launches": launches,
        "clocks": clk,
        "stable": stable,
    }
    if near is not None:
        line["near_field_vs_fraunhofer"] = near
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(w, budget_s=args.cpu_budget)
    if ws > 1:
        dist.destroy_process_group()
    return line


def run_cyl(args):
    """The paper's 2D axisymmetric solver on an n x n grid (Table I sizes),
    n steps by default, 64 detectors, the paper's Gaussian shower."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    import paper_1001_5341_gb300 as fd

    n = args.n
    w = W.cyl_table1(n, seed=4004 + rank)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g = fd.Cylinder(w.nr, w.nz, w.d, w.dt, w.eps_r, w.boundary, stream=stream)
        if args.cyl_kernel >= 0 or args.seg_rows > 0:
            g.set_kernel(args.cyl_kernel if args.cyl_kernel >= 0 else g.kernel_info["kernel"], args.seg_rows)
        K = g.kernel_info["steps_per_launch"]
        steps = args.steps if args.steps else n
        steps = max(K, steps // K * K)
        q_tab, ring_w = fd.cyl_tables(w)
        g.set_shower(q_tab, w.z0, w.bin_dz, w.v, ring_w)
        tune_max = 48 * 2 * K                      # cyl_tune's bound on its steps (2 launches per length)
        g.set_probes(w.probes_rz, tune_max + args.warmup * K + steps)
        # segment length by timing real steps (untimed, before the warm-up),
        # unless a length was given
        tuned = g.tune(2) if args.seg_rows == 0 and not args.no_cyl_tune else 0
        info = g.kernel_info
        g.step(args.warmup * K)
        g.sync()
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.3)
        l0 = g.launches
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        g.step(steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        launches = g.launches - l0
        clk = clocks.stop()
        g.sync()
        # spectra of every detector's whole trace (Sec. V) through the C ABI,
        # timed on the same stream
        trd = torch.empty((w.probes_rz.shape[0], tune_max + args.warmup * K + steps, 2), dtype=torch.float32,
                          device="cuda")
        g.probes(out=trd)
        trd = trd[:, :tuned + args.warmup * K + steps].contiguous()   # the steps done
        freqs = np.linspace(10e6, 2e9, 1024)
        th = np.full(trd.shape[0], math.acos(1 / math.sqrt(w.eps_r)))
        fd.trace_spectrum(trd, w.dt, freqs, t0=w.dt, coef=fd.theta_coef(th), stream=stream)
        ev0.record(stream)
        fd.trace_spectrum(trd, w.dt, freqs, t0=w.dt, coef=fd.theta_coef(th), stream=stream)
        ev1.record(stream)
        torch.cuda.synchronize()
        spec_ms = ev0.elapsed_time(ev1)
        spec_terms = trd.shape[0] * trd.shape[1] * freqs.size
        del trd
        # end to end with host buffers
        q, wr, rz = (np.ascontiguousarray(a) for a in (q_tab, ring_w, w.probes_rz))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.reset()
        g.set_shower(q, w.z0, w.bin_dz, w.v, wr)
        g.set_probes(rz, steps)
        g.step(steps)
        tr = g.probes()
        e2e_s = time.perf_counter() - t0
        g.close()
    if rank != 0:
        return None
    cells = w.cells
    value = ws * cells * steps / (ms * 1e-3) / 1e9
    peak, peak_kind = hbm_peak()
    comp_cells = 3 * cells + w.nr + w.nz                  # E_r, E_z, H_phi
    bytes_launch = 8.0 * comp_cells if K > 1 else 36.0 * cells / 1.0
    n_launch = steps // K if K > 1 else steps
    achieved = bytes_launch * n_launch / (ms * 1e-3) / 1e9
    kname = info["kernel_name"]
    fset = 2 * 3 * (w.nr + 1) * ((w.nz + 1 + 16 + 63) // 32 * 32) * 4 / 1e9
    line = {
        "metric": "Gcell-updates/s", "value": round(value, 3), "unit": "Gcell/s", "solver": "cyl2d",
        "n_gpus": ws, "steps": steps, "warmup": args.warmup * K,
        "ms_per_step": round(ms / steps, 6), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**w.describe(), "seed": 4004, **info, "tuning_steps": tuned,
                   "inputs_vs_l2": f"fields {fset:.3f} GB vs 129 MB L2 (no flush: one timed call)"},
        "roofline": {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": round(achieved / peak, 4),
                     "bytes_per_launch_alg": bytes_launch, "steps_per_launch": K,
                     "traffic": (ncu_record(kname, w.name) or {}).get("dram_bytes_per_launch"),
                     "single_step_equiv_GBps": round(24.0 * value, 1)},
        "e2e": {"value": round(ws * cells * steps / e2e_s / 1e9, 3), "unit": "Gcell/s",
                "h2d_bytes_per_step": round((q.nbytes + wr.nbytes + rz.nbytes) / steps, 2),
                "d2h_bytes_per_step": round(tr.nbytes / steps, 2),
                "what": "reset + set_shower + set_probes (host tables) + step(n) + probes() to host"},
        "gpu_launches": launches, "clocks": clk,
        "paper_table1_t_gpu_s": PAPER_T_GPU.get(n),
        "spectrum": {"kernel": "k_trace_spectrum", "traces": int(w.probes_rz.shape[0]),
                     "samples": int(spec_terms // (w.probes_rz.shape[0] * 1024)), "freqs": 1024,
                     "ms": round(spec_ms, 3), "G_sample_freq_per_s": round(spec_terms / (spec_ms * 1e-3) / 1e9, 2),
                     "what": "theta-hat E_omega of every detector's whole trace, one fdtd_trace_spectrum call"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cyl_cpu_baseline(w, budget_s=args.cpu_budget)
    return line


ADJ_GRID = (256, 256, 512)


def adjoint_problem(fd, TraceModel, rank=0, steps=2000, stream=None):
    """The adjoint workload (seed 5005 + rank): a 256 x 256 x 512 PEC grid,
    dx = 2 cm, a 256-bin Gaussian charge table (l = 1.2 m), Gaussian lateral
    spread (L = 4), 64 detectors at r = 0.5-2.2 m.  Returns the simulation,
    the differentiable trace model over `steps` steps, and the table."""
    nx, ny, nz = ADJ_GRID
    dx = 0.02
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    rng = np.random.default_rng(5005 + rank)
    n_bins, z0 = 256, 0.2
    bin_dz = (nz * dx) / n_bins
    q = fd.profile_gaussian(z0, bin_dz, n_bins, 4.0 + rng.random(), 1.2, -1e-9)
    lw = fd.lateral_gaussian(4, 1.0)
    cx, cy = nx // 2 * dx, ny // 2 * dx
    r = rng.uniform(0.5, 2.2, 64)
    ph = rng.uniform(0, 2 * np.pi, 64)
    xyz = np.stack([cx + r * np.cos(ph), cy + r * np.sin(ph), rng.uniform(1.0, nz * dx - 1.0, 64)], axis=1)
    kw = {} if stream is None else {"stream": stream}
    sim = fd.Simulation(nx, ny, nz, dx, dt, W.EPS_R_ICE, boundary=fd.FDTD_PEC, **kw)
    sim.set_probes(xyz, steps)
    return sim, TraceModel(sim, z0, bin_dz, W.C0, lw, 4, steps), q


def run_adjoint(args):
    """Gradient of a detector misfit with respect to a 256-bin charge table on
    a 256 x 256 x 512 PEC grid (dx = 2 cm): the forward run and the adjoint
    run, each timed on the device."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    import paper_1001_5341_gb300 as fd
    from paper_1001_5341_gb300.adjoint import TraceModel

    nx, ny, nz = ADJ_GRID
    steps = args.steps or 2000
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim, model, q = adjoint_problem(fd, TraceModel, rank, steps, stream=stream)
        qt = torch.tensor(q, requires_grad=True)
        with torch.no_grad():
            target = model(qt * 0.9)
        # untimed warm-up of the whole forward + loss + backward path: the
        # first autograd backward of a process loads torch's kernels
        yw = model(qt)
        (0.5 * ((yw.double() - target.double()) ** 2).sum()).backward()
        qt.grad = None
        clocks = ClockSampler(local)
        clocks.start()
        time.sleep(0.5)   # the sampler's start-up stalls the driver for a moment
        # both passes end in a synchronisation inside the library (traces to
        # the tensor, gradient to the host): synchronised wall clocks
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        y = model(qt)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        loss = 0.5 * ((y.double() - target.double()) ** 2).sum()
        loss.backward()
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        clk = clocks.stop()
        t_fwd, t_all = t1 - t0, t2 - t0
        launches = sim.launches
        g = qt.grad.numpy()
        sim.close()
    if rank != 0:
        return None
    cells = nx * ny * nz
    t_adj = t_all - t_fwd
    return {"metric": "gradient evaluations/s", "value": round(1.0 / t_all, 4), "unit": "gradients/s",
            "solver": "adjoint", "n_gpus": ws, "steps": steps, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"pec{nx}x{ny}x{nz}", "dx_m": 0.02, "bins": int(q.size), "probes": 64,
                       "lateral_L": 4, "loss": "1/2 sum (traces - traces(0.9 q))^2"},
            "forward_s": round(t_fwd, 4), "adjoint_s": round(t_adj, 4),
            "forward_gcells": round(cells * steps / t_fwd / 1e9, 2),
            "adjoint_gcells": round(cells * steps / t_adj / 1e9, 2),
            "adjoint_over_forward": round(t_adj / t_fwd, 3),
            "grad_norm": float(np.linalg.norm(g)), "gpu_launches": launches, "clocks": clk}


BATCH_DX = 0.02


def batch_workload(fd, kind="config4", rank=0, max_steps=1800):
    """Grid sizes and a constructor of the batch workloads (seed 6006 + rank):
    "config4" = 64 showers on 64^3 .. 256 x 256 x 512, "small" = 256 showers
    on 32^3 .. 96^3; dx = 2 cm, Mur, Gaussian profile and lateral spread, 8
    detectors each.  make(dims, seed) returns a Simulation with trace room
    for max_steps steps."""
    rng = np.random.default_rng(6006 + rank)
    dx = BATCH_DX
    dt = W.courant_dt(dx, W.EPS_R_ICE)
    if kind == "small":
        dims = [tuple(int(v) for v in rng.integers(32, 97, 3)) for _ in range(256)]
    else:
        dims = [(int(rng.integers(64, 257)), int(rng.integers(64, 257)), int(rng.integers(64, 513)))
                for _ in range(64)]
    lw = fd.lateral_gaussian(3, 1.0)

    def make(d, seed):
        r = np.random.default_rng(seed)
        nx, ny, nz = d
        sim = fd.Simulation(nx, ny, nz, dx, dt, W.EPS_R_ICE, boundary=fd.FDTD_MUR1)
        nb, z0 = 128, 0.0
        bdz = nz * dx / (nb - 1)
        q = fd.profile_gaussian(z0, bdz, nb, r.uniform(0.3, 0.7) * nz * dx, r.uniform(0.1, 0.3) * nz * dx, -1e-9)
        sim.set_shower(q, z0, bdz, W.C0, lw, 3)
        cx, cy = nx // 2 * dx, ny // 2 * dx
        rr = r.uniform(0.2, 0.4, 8) * min(nx, ny) * dx
        ph = r.uniform(0, 2 * np.pi, 8)
        xyz = np.stack([cx + rr * np.cos(ph), cy + rr * np.sin(ph), r.uniform(0.2, 0.8, 8) * nz * dx], 1)
        sim.set_probes(xyz, max_steps)
        return sim

    return dims, make


def run_batch(args):
    """64 independent showers on uneven grids (64^3 .. 256 x 256 x 512, dx =
    2 cm, Mur) advanced together by one batch (the persistent kernel and the
    solo streams, as its autotuner chooses; then each way alone), against the
    same simulations stepped one after another (default one-pass tile path,
    and the unfused path)."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    import paper_1001_5341_gb300 as fd

    steps = args.steps or 200
    dims, make = batch_workload(fd, args.batch_kind, rank, 4 * steps + 1000)
    n_sims = len(dims)
    dx = BATCH_DX
    sims = [make(d, 7000 + i) for i, d in enumerate(dims)]
    cells = sum(nx * ny * nz for nx, ny, nz in dims)

    def timed(fn):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn()
        torch.cuda.synchronize()
        return time.perf_counter() - t0

    b = fd.Batch(sims)
    if args.chunk_planes:
        b.set_config(args.chunk_planes, 8)
    if args.batch_mode == "tuned":
        used = b.tune(trial_steps=2)
    else:
        used = 0
        b.set_solo(-1 if args.batch_mode == "persistent" else 1)
    b.step(args.warmup)
    b.sync()
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.5)
    t_batch = timed(lambda: (b.step(steps), b.sync()))
    clk = clocks.stop()
    cfg, graph, solo = b.config, b.graph_mode, b.solo
    g = lambda t: round(cells * steps / t / 1e9, 2)
    extra = {}
    if args.batch_mode == "tuned":
        # each way alone: every grid in the persistent kernel, every grid on
        # the solo streams
        ways = {}
        for name, thr in (("persistent_only", -1), ("solo_streams_only", 1)):
            b.set_solo(thr)
            b.step(2)
            b.sync()
            ways[name] = timed(lambda: (b.step(steps), b.sync()))
        b.set_solo(solo["min_cells"])
        t_fused = timed(lambda: [s.step(steps) for s in sims])
        for s in sims:
            s.set_kernel(0)
        t_unfused = timed(lambda: [s.step(steps) for s in sims])
        extra = {"persistent_only_gcells": g(ways["persistent_only"]),
                 "solo_streams_only_gcells": g(ways["solo_streams_only"]),
                 "one_by_one_fused_gcells": g(t_fused), "one_by_one_unfused_gcells": g(t_unfused),
                 "batch_over_fused": round(t_fused / t_batch, 3), "batch_over_unfused": round(t_unfused / t_batch, 3)}
    b.close()
    for s in sims:
        s.close()
    if rank != 0:
        return None
    return {"metric": "Gcell-updates/s", "value": g(t_batch), "unit": "Gcell/s", "solver": "batch",
            "n_gpus": ws, "steps": steps, "warmup": args.warmup, "higher_is_better": True, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batch{n_sims}-uneven", "simulations": n_sims, "cells_total": cells,
                       "grids": ("nx, ny, nz in [32, 96]" if args.batch_kind == "small"
                                 else "nx, ny in [64, 256], nz in [64, 512]") + ", seeded", "boundary": "mur1",
                       "dx_m": dx, "probes_each": 8, **cfg, "graph_replay": bool(graph == 1),
                       "solo_min_cells": solo["min_cells"], "solo_grids": solo["n_solo"],
                       "tuner_trial_steps": used, "batch_mode": args.batch_mode},
            **extra, "clocks": clk}


def run_gemm(args):
    """The surrogate's bf16 GEMM (sur_gemm_bf16) on its two kernels: the
    tcgen05 kernel (TMEM accumulator, TMA-staged 128-byte-swizzled slices)
    and the mma.sync kernel.  Shapes: the lattice surrogate's serving product
    at one antenna (P profiles x T = 1024 samples x 96: [hi, hi, lo] x 31 bins
    padded to 96), whose output write makes it HBM-bound, and an 8192^3
    product for the kernels' tensor throughput.  CUDA events on the launching
    stream; the serving product rotates over outputs larger than L2."""
    import torch
    import ctypes as C
    torch.cuda.set_device(0)
    import paper_1001_5341_gb300 as fd
    peaks = {}
    try:
        with open(MEASURED_PEAKS) as f:
            peaks = json.load(f)
    except Exception:
        pass
    tf_peak = float(peaks.get("bf16_tflops", 1900.0))
    hbm, _ = hbm_peak()
    steps = args.steps or 50
    p = lambda t: C.c_void_p(t.data_ptr())
    g = torch.Generator(device="cuda").manual_seed(9009)
    res = {}

    def time_it(fn, n):
        for _ in range(3):
            fn(0)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(n):
            fn(i)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    for name, (M, N, K) in (("serving", (args.gemm_profiles, 1024, 96)), ("square", (8192, 8192, 8192))):
        A = torch.randn(M, K, generator=g, device="cuda").to(torch.bfloat16)
        B = torch.randn(N, K, generator=g, device="cuda").to(torch.bfloat16)
        nout = max(1, (256 << 20) // (M * N * 4)) if name == "serving" else 1
        Ys = [torch.empty(M, N, dtype=torch.float32, device="cuda") for _ in range(nout)]
        for path, label in ((0, "tcgen05"), (1, "mma_sync")):
            fd.check(fd.sur_gemm_set_path(path), "path")
            n0 = fd.sur_gemm_tc_launches()
            fn = lambda i: fd.check(fd.sur_gemm_bf16(p(A), K, 1, p(B), K, 1, p(Ys[i % nout]), N, None, M, N, K, None,
                                                     0, 0, None), "gemm")
            ms = time_it(fn, steps if name == "serving" else max(3, steps // 10))
            ran_tc = fd.sur_gemm_tc_launches() > n0
            flops = 2.0 * M * N * K
            byts = M * N * 4 + (M + N) * K * 2
            res[f"{name}_{label}"] = {"shape_MNK": [M, N, K], "ms": round(ms, 5),
                                      "tflops": round(flops / ms / 1e9, 2),
                                      "frac_of_bf16_peak": round(flops / ms / 1e9 / tf_peak, 4),
                                      "gbs": round(byts / ms / 1e6, 1), "frac_of_hbm": round(byts / ms / 1e6 / hbm, 4),
                                      "tcgen05_kernel": bool(ran_tc)}
        fd.check(fd.sur_gemm_set_path(0), "path")
        assert fd.sur_gemm_tc_failed() == 0
        del A, B, Ys
        torch.cuda.empty_cache()
    sv = res["serving_tcgen05"]
    return {"metric": "TFLOP/s", "value": sv["tflops"], "unit": "TFLOP/s", "solver": "gemm", "n_gpus": 1,
            "steps": steps, "higher_is_better": True, "dtype": "bf16", "data": "synthetic",
            "config": {"workload": f"surrogate-gemm-{args.gemm_profiles}x1024x96",
                       "inputs_vs_l2": "serving outputs rotate over > 256 MB"},
            "roofline": {"bound": "hbm", "achieved": sv["gbs"], "peak": hbm, "unit": "GB/s",
                         "frac": sv["frac_of_hbm"], "traffic": None},
            "bf16_peak_tflops": tf_peak, "kernels": res}


# Table I: GTX285 seconds per N^2 run (step count not printed; read as N steps)
PAPER_T_GPU = {256: 0.040, 512: 0.186, 1024: 1.167, 2048: 8.372, 4096: 67.617, 8192: 681.082}


def _cyl_oracle_shower(s):
    """set_shower arguments of the 2D oracle, its tables built by the oracle."""
    from oracle import cyl_oracle as CO
    q, rings = CO.tables(s)
    return q, s.z0, s.bin_dz, s.v, rings


def cyl_cpu_baseline(w, budget_s=15.0):
    """The 2D FP64 oracle as it stands, on a 1024 x 1024 sample of the same physics."""
    from oracle import cyl_oracle as CO
    m = min(1024, w.nr)
    s = W.cyl_table1(m, extent_m=w.d * m)
    o = CO.CylOracle(s.nr, s.nz, s.d, s.dt, s.eps_r, boundary=s.boundary)
    o.set_shower(*_cyl_oracle_shower(s))
    o.set_probes(s.probes_rz)
    o.step(1)
    done = 0
    t1 = time.perf_counter()
    while time.perf_counter() - t1 < budget_s:
        o.step(1)
        done += 1
    el = time.perf_counter() - t1
    return {"value": round(s.cells * done / el / 1e9, 6), "unit": "Gcell/s", "cores": _omp_threads(),
            "kind": "oracle", "sample": f"{m}x{m} cells, same d and shower model, {done} steps, {el:.1f} s"}


def _oracle_sample(w, target_cells):
    """The workload's physics (dx, dt, CPML, shower, lateral spread) on a
    sub-grid of about target_cells cells with the same aspect ratio, never
    larger than the workload's own grid."""
    f = min(1.0, (target_cells / w.cells) ** (1.0 / 3.0))
    min_n = 2 * w.npml + 8
    # the lateral footprint (+-L cells about the axis) must stay clear of the CPML
    min_xy = max(min_n, 2 * (w.npml + 1 + int(w.lateral.get("L", 0))) + 2)
    nx = min(w.nx, max(min_xy, int(w.nx * f) // 2 * 2))
    ny = min(w.ny, max(min_xy, int(w.ny * f) // 2 * 2))
    nz = min(w.nz, max(min_n, int(w.nz * f) // 2 * 2))
    r_hi = min(0.3, (min(nx, ny) // 2 - w.npml - 2) * w.dx * 0.9)
    if w.profile["kind"] == "gh":
        # subshowers spread over the sample's own length
        spread = min(40.0, max(0.0, (nz - 2 * w.npml - 8) * w.dx - 6.0))   # 40 m: the workload's own
        return W.gh640(nx=nx, ny=ny, nz=nz, npml=w.npml, steps=1, n_probes=8, r_lo=0.1, r_hi=r_hi,
                       spread_m=spread)
    return W.greisen384(nx=nx, ny=ny, nz=nz, npml=w.npml, steps=1, n_probes=8,
                        r_lo=0.1, r_hi=r_hi, E0=w.profile["E0_eV"])


def _shower_text(w):
    if w.profile["kind"] == "gh":
        return f"{len(w.profile['z1'])} Gaisser-Hillas subshowers, dx {w.dx * 100:.0f} cm"
    return f"Greisen E0={w.profile['E0_eV']:.3g} eV"


def _omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def cpu_baseline(w, budget_s=15.0):
    """The FP64 oracle as it stands, on the host cores, over a bounded sample."""
    import oracle
    t0 = time.perf_counter()
    sw = _oracle_sample(w, 4.0e6)
    o = oracle.from_workload(sw, max_steps=100000)
    o.step(1)
    done = 0
    t1 = time.perf_counter()
    while True:
        o.step(1)
        done += 1
        if time.perf_counter() - t1 > budget_s:
            break
    el = time.perf_counter() - t1
    cores = oracle.set_threads(0)
    # the same oracle on one thread, as the paper's sequential CPU code ran
    oracle.set_threads(1)
    done1 = 0
    t2 = time.perf_counter()
    while True:
        o.step(1)
        done1 += 1
        if time.perf_counter() - t2 > budget_s / 3:
            break
    el1 = time.perf_counter() - t2
    oracle.set_threads(cores)
    return {"value": round(sw.cells * done / el / 1e9, 5), "unit": "Gcell/s", "cores": cores,
            "kind": "oracle",
            "sample": f"{sw.nx}x{sw.ny}x{sw.nz} cells of the same physics (CPML {sw.npml}, {_shower_text(w)}, "
                      f"NKG lateral), {done} steps, "
                      f"{el:.1f} s (setup {t1 - t0:.1f} s excluded)",
            "single_thread": {"value": round(sw.cells * done1 / el1 / 1e9, 5), "unit": "Gcell/s",
                              "sample": f"the same grid, {done1} more steps on one thread, {el1:.1f} s"}}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    import oracle
    w = replica_workload(0, args.workload)
    # size the per-step sample so that W + K oracle steps take about two minutes
    cal = _oracle_sample(w, 2.0e5)
    o = oracle.from_workload(cal, max_steps=100)
    o.step(1)
    t = time.perf_counter()
    o.step(3)
    rate = 3 * cal.cells / (time.perf_counter() - t)
    del o
    per_step_s = min(2.0, 120.0 / max(1, args.steps + args.warmup))
    sw = _oracle_sample(w, max(5e4, rate * per_step_s))
    o = oracle.from_workload(sw, max_steps=args.warmup + args.steps)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(args.steps)
    el = time.perf_counter() - t0
    v = sw.cells * args.steps / el / 1e9
    sample = (f"each step: one oracle step on {sw.nx}x{sw.ny}x{sw.nz} cells of the same physics "
              f"(CPML {sw.npml}, {_shower_text(sw)}, NKG lateral)")
    return {"impl": "reference", "metric": "Gcell-updates/s", "value": round(v, 6), "unit": "Gcell/s",
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(el * 1e3 / args.steps, 4), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {**w.describe(), "seed": WORKLOAD_SEEDS[args.workload]},
            "cpu_baseline": {"value": round(v, 6), "unit": "Gcell/s", "cores": _omp_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "Gcell/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def run_cyl_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return None
    from oracle import cyl_oracle as CO
    n = args.n
    w = W.cyl_table1(n)
    m = min(512, n)
    s = W.cyl_table1(m, extent_m=w.d * m)
    steps = args.steps or 64
    o = CO.CylOracle(s.nr, s.nz, s.d, s.dt, s.eps_r, boundary=s.boundary)
    o.set_shower(*_cyl_oracle_shower(s))
    o.set_probes(s.probes_rz)
    o.step(args.warmup)
    t0 = time.perf_counter()
    o.step(steps)
    el = time.perf_counter() - t0
    v = s.cells * steps / el / 1e9
    sample = f"each step: one oracle step on {m}x{m} cells of the same d and shower model"
    return {"impl": "reference", "solver": "cyl2d", "metric": "Gcell-updates/s", "value": round(v, 6),
            "unit": "Gcell/s", "n_gpus": ws, "steps": steps, "warmup": args.warmup,
            "ms_per_step": round(el * 1e3 / steps, 4), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": w.describe(),
            "cpu_baseline": {"value": round(v, 6), "unit": "Gcell/s", "cores": _omp_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(v, 6), "unit": "Gcell/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: 1000 for yee3d, n for cyl)")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--nz", type=int, default=0,
                    help="z planes of a reduced grid with the benchmark physics (profiler captures "
                         "of a few GB); 0 = the benchmark grid")
    ap.add_argument("--solver", choices=["yee3d", "cyl", "adjoint", "batch", "gemm"], default="yee3d",
                    help="cyl: the paper's 2D axisymmetric solver on an n x n grid (Table I); "
                         "adjoint: gradient of a detector misfit w.r.t. the charge table")
    ap.add_argument("--workload", choices=sorted(WORKLOAD_SEEDS), default="greisen384",
                    help="3D workload: greisen384 (384x384x1536, the headline) or gh640 (640x640x2048, dx 3 cm)")
    ap.add_argument("--n", type=int, default=8192, help="cyl grid side")
    ap.add_argument("--cyl-kernel", type=int, default=-1, help="cyl kernel (-1: library default)")
    ap.add_argument("--kernel", type=int, default=-1,
                    help="3D field-update path (fdtd_set_kernel; -1: library default)")
    ap.add_argument("--batch-mode", choices=["tuned", "persistent", "solo"], default="tuned",
                    help="batch: the autotuner's choice (with each way alone and one by one for comparison), "
                         "or only the persistent kernel, or only the solo streams")
    ap.add_argument("--chunk-planes", type=int, default=0, help="batch: z planes per tile item (0: default)")
    ap.add_argument("--batch-kind", choices=["config4", "small"], default="config4",
                    help="batch workload: 64 grids 64^3 .. 256x256x512, or 256 grids 32^3 .. 96^3")
    ap.add_argument("--seg-rows", type=int, default=0, help="cyl rows per segment (0: tuned by cyl_tune)")
    ap.add_argument("--no-cyl-tune", action="store_true", help="cyl: keep the library's segment model")
    ap.add_argument("--gemm-profiles", type=int, default=8192, help="gemm: profiles of the serving product")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.solver == "adjoint":
        line = run_adjoint(args)
    elif args.solver == "batch":
        line = run_batch(args)
    elif args.solver == "gemm":
        line = run_gemm(args)
    elif args.solver == "cyl":
        if args.impl == "reference":
            line = run_cyl_reference(args)
        else:
            line = run_cyl(args)
    else:
        if not args.steps:
            args.steps = 1000
        line = run_reference(args) if args.impl == "reference" else run_ours(args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
