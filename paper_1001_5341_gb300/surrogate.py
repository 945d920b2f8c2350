"""Learned near-field surrogate: maps a shower's longitudinal charge profile
and an antenna position to the Ez pulse there, trained on traces of the FDTD
path (fdtd_* calls); FDTD stays the reference and the fallback.  The paper
has no counterpart to this module.

Structure.  The trace is linear in the binned profile q_k (the field
equations are linear in the current), and in a uniform medium the response of
bin k depends only on the antenna's radius r, its axial offset dz_k = z_a -
z_k and the time since the shower front reached the bin.  Bins are m shower
steps long, so that time is a whole number of samples (shift k):

    trace[i] = peak|q| c_out sum_k qn_k (1/R_k) G(r, dz_k)(i - shift k - R_k/c')

Each bin's response is placed in its own retarded time, shifted by the
direct travel time R_k / c' from the bin to the antenna (linear interpolation
between samples) and scaled by 1/R_k, so the network only learns a smooth
shape: G(r, dz) is a waveform of Tg samples (J0 before the direct arrival)
from an MLP on 64 features of (r, dz) (64 -> H -> H -> Tg, ReLU between),
the learned counterpart of the Green's function superposition of Sec. II.
The sum over bins is a 1D transposed convolution along the shower.

Every arithmetic step runs in the library's CUDA kernels (surrogate.h):
bf16 tensor-core GEMMs (f32 accumulation), the bin assembly and its
gradient, ReLU, MSE, Adam, input scaling and features.  PyTorch only
allocates device memory and supplies the stream.
"""
from __future__ import annotations

import ctypes as C
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import (check, fdtd_probes, profile_gaisser_hillas, lateral_nkg, Simulation, sur_adam, sur_antenna_features,
               sur_assemble, sur_assemble_bwd, sur_bias_grad, sur_cast_bf16, sur_gemm_bf16, sur_lattice_bwd,
               sur_gemm_bf16_batched, sur_lattice_fwd, sur_lattice_fwd_f32, sur_lattice_weights,
               sur_lattice_weights_kmajor, sur_mse,
               sur_normalize_rows, sur_pairs, sur_relu_bwd, sur_scale_rows, sur_split3_bf16, sur_split_bf16)

N_FEAT = 64


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@dataclass
class Geometry:
    """Profile bins and trace sampling shared by the data and the network."""
    K: int = 128            # profile bins
    z0: float = 0.28        # axial position of bin 0 (metres)
    dz: float = 0.0822      # bin length (metres) = m v dt
    shift: int = 4          # trace samples between the passages of consecutive bins
    T: int = 1024           # trace samples
    Tg: int = 1024          # samples of one bin's response
    cps: float = 0.01187    # metres the wave covers per trace sample (c/n x sample time)
    J0: int = 16            # response samples before the direct arrival
    feat: tuple = (0.6, 0.3, 0.0, 10.5)   # (r0, rs, z0, zs) of the (r, dz) features

    @classmethod
    def of(cls, grid, decim: int, m: int, **kw):
        """Bins of m steps of the shower on `grid` (workloads.surrogate_grid),
        traces every `decim` steps (m a multiple of decim)."""
        assert m % decim == 0
        cps = 299792458.0 / math.sqrt(grid.eps_r) * grid.dt * decim
        return cls(K=grid.n_bins, z0=grid.z0, dz=grid.bin_dz, shift=m // decim, T=grid.steps // decim,
                   Tg=grid.steps // decim, cps=cps, **kw)


class Net:
    """Parameters (f32 master, bf16 copy, gradient, Adam moments) on the
    current CUDA device, and the forward / backward / step kernels."""

    def __init__(self, geom: Geometry, hidden: int = 1024, seed: int = 0, c_out: float = 1.0):
        import torch
        self.geo = geom
        self.H = hidden
        self.c_out = float(c_out)
        self.t = 0
        rng = np.random.default_rng(seed)
        self.p, self.pb, self.g, self.m, self.v = {}, {}, {}, {}, {}
        for i, (fin, fout) in enumerate(((N_FEAT, hidden), (hidden, hidden), (hidden, geom.Tg))):
            lim = math.sqrt(6.0 / fin) if i < 2 else math.sqrt(3.0 / fin)
            for name, shp, w0 in ((f"f{i}w", (fout, fin), rng.uniform(-lim, lim, size=(fout, fin))),
                                  (f"f{i}b", (fout,), np.zeros(fout))):
                self.p[name] = torch.tensor(w0, dtype=torch.float32, device="cuda")
                self.g[name] = torch.zeros(shp, dtype=torch.float32, device="cuda")
                self.m[name] = torch.zeros(shp, dtype=torch.float32, device="cuda")
                self.v[name] = torch.zeros(shp, dtype=torch.float32, device="cuda")
                if name.endswith("w"):
                    self.pb[name] = torch.empty(shp, dtype=torch.bfloat16, device="cuda")
                    check(sur_cast_bf16(_p(self.p[name]), _p(self.pb[name]), self.p[name].numel(), _stream()),
                          "sur_cast_bf16")
        self._ws = {}

    @property
    def n_params(self) -> int:
        return sum(t.numel() for t in self.p.values())

    def _workspace(self, B):
        import torch
        if B in self._ws:
            return self._ws[B]
        g, H = self.geo, self.H
        BK = B * g.K
        f32, b16 = torch.float32, torch.bfloat16
        e = lambda *s, dt=f32: torch.empty(s, dtype=dt, device="cuda")
        w = {"qn": e(B, g.K), "s": e(B), "pairs": e(BK, 2), "feat": e(BK, N_FEAT), "featb": e(BK, N_FEAT, dt=b16),
             "h1": e(BK, H), "h1b": e(BK, H, dt=b16), "h2": e(BK, H), "h2b": e(BK, H, dt=b16), "G": e(BK, g.Tg),
             "y": e(B, g.T), "tn": e(B, g.T), "dy": e(B, g.T), "dG": e(BK, g.Tg), "dGb": e(BK, g.Tg, dt=b16),
             "dh2": e(BK, H), "dz2": e(BK, H), "dz2b": e(BK, H, dt=b16),
             "dh1": e(BK, H), "dz1": e(BK, H), "dz1b": e(BK, H, dt=b16), "loss": e(1)}
        self._ws = {B: w}   # keep one batch size resident
        return w

    def forward(self, q, rz, scale_out=True):
        """Traces [B, T] (f32, device) for profiles q [B, K] (C per bin) and
        antenna positions rz [B, 2] (metres), both device f32.  With
        scale_out=False: the normalised trace (trace / (peak|q| c_out))."""
        B = q.shape[0]
        g, H = self.geo, self.H
        BK = B * g.K
        w = self._workspace(B)
        st = _stream()
        check(sur_normalize_rows(_p(q), B, g.K, _p(w["qn"]), _p(w["s"]), st), "sur_normalize_rows")
        check(sur_pairs(_p(rz), B, g.K, g.z0, g.dz, _p(w["pairs"]), st), "sur_pairs")
        check(sur_antenna_features(_p(w["pairs"]), BK, *g.feat, _p(w["feat"]), st), "sur_antenna_features")
        check(sur_cast_bf16(_p(w["feat"]), _p(w["featb"]), BK * N_FEAT, st), "sur_cast_bf16")
        check(sur_gemm_bf16(_p(w["featb"]), N_FEAT, 1, _p(self.pb["f0w"]), N_FEAT, 1, _p(w["h1"]), H, _p(w["h1b"]),
                            BK, H, N_FEAT, _p(self.p["f0b"]), 1, 0, st), "sur_gemm_bf16")
        check(sur_gemm_bf16(_p(w["h1b"]), H, 1, _p(self.pb["f1w"]), H, 1, _p(w["h2"]), H, _p(w["h2b"]),
                            BK, H, H, _p(self.p["f1b"]), 1, 0, st), "sur_gemm_bf16")
        check(sur_gemm_bf16(_p(w["h2b"]), H, 1, _p(self.pb["f2w"]), H, 1, _p(w["G"]), g.Tg, None,
                            BK, g.Tg, H, _p(self.p["f2b"]), 0, 0, st), "sur_gemm_bf16")
        check(sur_assemble(_p(w["G"]), _p(w["qn"]), _p(rz), B, g.K, g.Tg, g.shift, g.T, g.z0, g.dz, g.cps, g.J0,
                           _p(w["y"]), st), "sur_assemble")
        w["rz"] = rz
        if scale_out:
            check(sur_scale_rows(_p(w["y"]), B, g.T, _p(w["s"]), self.c_out, 0, st), "sur_scale_rows")
        return w["y"]

    def backward(self, B):
        """Gradients of the MSE between the normalised output and w['tn'];
        returns the device loss tensor (f32[1])."""
        g, H = self.geo, self.H
        BK = B * g.K
        w = self._workspace(B)
        st, G, pb = _stream(), self.g, self.pb
        check(sur_mse(_p(w["y"]), _p(w["tn"]), B * g.T, _p(w["dy"]), _p(w["loss"]), st), "sur_mse")
        check(sur_assemble_bwd(_p(w["dy"]), _p(w["qn"]), _p(w["rz"]), B, g.K, g.Tg, g.shift, g.T, g.z0, g.dz, g.cps,
                               g.J0, _p(w["dG"]), _p(w["dGb"]), st), "sur_assemble_bwd")
        # output layer: G = h2b W2^T + b2
        check(sur_gemm_bf16(_p(w["dGb"]), g.Tg, 0, _p(w["h2b"]), H, 0, _p(G["f2w"]), H, None, g.Tg, H, BK, None, 0,
                            0, st), "sur_gemm_bf16")
        check(sur_bias_grad(_p(w["dG"]), g.Tg, BK, g.Tg, _p(G["f2b"]), st), "sur_bias_grad")
        check(sur_gemm_bf16(_p(w["dGb"]), g.Tg, 1, _p(pb["f2w"]), H, 0, _p(w["dh2"]), H, None, BK, H, g.Tg, None, 0,
                            0, st), "sur_gemm_bf16")
        check(sur_relu_bwd(_p(w["h2"]), _p(w["dh2"]), _p(w["dz2"]), _p(w["dz2b"]), BK * H, st), "sur_relu_bwd")
        # hidden layer 1
        check(sur_gemm_bf16(_p(w["dz2b"]), H, 0, _p(w["h1b"]), H, 0, _p(G["f1w"]), H, None, H, H, BK, None, 0, 0,
                            st), "sur_gemm_bf16")
        check(sur_bias_grad(_p(w["dz2"]), H, BK, H, _p(G["f1b"]), st), "sur_bias_grad")
        check(sur_gemm_bf16(_p(w["dz2b"]), H, 1, _p(pb["f1w"]), H, 0, _p(w["dh1"]), H, None, BK, H, H, None, 0, 0,
                            st), "sur_gemm_bf16")
        check(sur_relu_bwd(_p(w["h1"]), _p(w["dh1"]), _p(w["dz1"]), _p(w["dz1b"]), BK * H, st), "sur_relu_bwd")
        # hidden layer 0
        check(sur_gemm_bf16(_p(w["dz1b"]), H, 0, _p(w["featb"]), N_FEAT, 0, _p(G["f0w"]), N_FEAT, None, H, N_FEAT, BK,
                            None, 0, 0, st), "sur_gemm_bf16")
        check(sur_bias_grad(_p(w["dz1"]), H, BK, H, _p(G["f0b"]), st), "sur_bias_grad")
        return w["loss"]

    def step(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        st = _stream()
        for name, wt in self.p.items():
            wb = _p(self.pb[name]) if name in self.pb else None
            check(sur_adam(_p(wt), wb, _p(self.g[name]), _p(self.m[name]), _p(self.v[name]), wt.numel(), lr, b1,
                           b2, eps, self.t, st), "sur_adam")

    def train_batch(self, q, rz, trace, lr):
        """One optimiser step on a batch (device tensors); returns the loss
        tensor (device)."""
        B = q.shape[0]
        w = self._workspace(B)
        self.forward(q, rz, scale_out=False)
        w["tn"].copy_(trace)
        check(sur_scale_rows(_p(w["tn"]), B, self.geo.T, _p(w["s"]), 1.0 / self.c_out, 1, _stream()),
              "sur_scale_rows")
        loss = self.backward(B)
        self.step(lr)
        return loss

    def predict(self, q, rz, chunk: int = 512):
        """Traces for many antennas, in chunks of `chunk` (device tensors)."""
        import torch
        out = torch.empty(q.shape[0], self.geo.T, dtype=torch.float32, device="cuda")
        for lo in range(0, q.shape[0], chunk):
            hi = min(q.shape[0], lo + chunk)
            out[lo:hi].copy_(self.forward(q[lo:hi].contiguous(), rz[lo:hi].contiguous()))
        return out


# ---- data from the FDTD path -------------------------------------------------

@dataclass
class Dataset:
    q: object          # [N, 128] f32 device: the profile table given to the FDTD run
    rz: object         # [N, 2] f32 device: antenna (r, z) in metres (snapped node)
    trace: object      # [N, T] f32 device: Ez, every `decim`-th step
    fdtd_s: float = 0.0           # wall time of the FDTD runs
    pulses_per_run: int = 0
    meta: dict = field(default_factory=dict)


def generate(grid, runs, decim: int = 2, log=None) -> Dataset:
    """Run the FDTD path once per entry of `runs` (workloads.surrogate_runs)
    on `grid` (workloads.surrogate_grid) and collect every detector's Ez
    trace.  One run gives all its detectors (Sec. III.B)."""
    import torch
    n_probes = runs[0]["probes_xyz"].shape[0]
    steps = grid.steps
    T = steps // decim
    N = len(runs) * n_probes
    q_all = torch.empty(N, grid.n_bins, dtype=torch.float32, device="cuda")
    rz_all = torch.empty(N, 2, dtype=torch.float32, device="cuda")
    tr_all = torch.empty(N, T, dtype=torch.float32, device="cuda")
    lw = lateral_nkg(grid.lateral["L"], grid.dx, grid.lateral["r_moliere"], grid.lateral["age"],
                     grid.lateral["nsub"], grid.lateral["r_cut"])
    sim = Simulation(grid.nx, grid.ny, grid.nz, grid.dx, grid.dt, grid.eps_r, grid.boundary, grid.npml)
    buf = torch.empty(n_probes, steps, 2, dtype=torch.float32, device="cuda")
    ic, jc = grid.nx // 2, grid.ny // 2
    t_fdtd = 0.0
    for r, run in enumerate(runs):
        q = profile_gaisser_hillas(grid.z0, grid.bin_dz, grid.n_bins, run["z1"], run["zmax"], run["lam"],
                                   run["nmax"], grid.profile["frac"])
        sim.reset()
        sim.set_shower(q, grid.z0, grid.bin_dz, grid.v, lw, grid.lateral["L"])
        sim.set_probes(run["probes_xyz"], steps)
        nodes = sim.probe_nodes()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.step(steps)
        check(fdtd_probes(sim.h, _p(buf), 1), "fdtd_probes")
        torch.cuda.synchronize()
        t_fdtd += time.perf_counter() - t0
        lo = r * n_probes
        tr_all[lo:lo + n_probes].copy_(buf[:, decim - 1::decim, 0])
        rr = np.hypot((nodes[:, 0] - ic) * grid.dx, (nodes[:, 1] - jc) * grid.dx)
        zz = nodes[:, 2] * grid.dx
        rz_all[lo:lo + n_probes].copy_(torch.tensor(np.stack([rr, zz], 1), dtype=torch.float32))
        q_all[lo:lo + n_probes].copy_(torch.tensor(q, dtype=torch.float32).expand(n_probes, -1))
        if log and (r + 1) % max(1, len(runs) // 10) == 0:
            log(f"fdtd run {r + 1}/{len(runs)}: {t_fdtd / (r + 1):.3f} s per run")
    sim.close()
    return Dataset(q_all, rz_all, tr_all, t_fdtd, n_probes,
                   {"grid": grid.describe(), "runs": len(runs), "decim": decim})


def rel_l2(pred, ref):
    """Per-sample relative L2 error ||pred - ref|| / ||ref|| of host arrays
    [N, T] (evaluation only)."""
    pred = np.asarray(pred, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return np.linalg.norm(pred - ref, axis=1) / np.maximum(np.linalg.norm(ref, axis=1), 1e-300)


# ---- lattice surrogate --------------------------------------------------------
#
# The lattice model drops the retarded-time interpolation of `Net`: on the grid
# of workloads.surrogate_lattice_grid (c dt = dx/2, bins of 4 cells = 8 steps)
# the field of bin k at an antenna is exactly the field of bin 0 at the antenna
# moved 4k cells back, 4k samples (8k steps) earlier.  For antennas on the
# lattice of workloads.surrogate_lattice_antennas (radial class ir, bin index
# m) the model is therefore
#     trace[t] = peak|q| c_out sum_k qn_k G[ir][m - k + moff][t - S k + J],
# (J = S lead samples: with the profile interpolated linearly between bins,
# bin k's charge starts to move one bin early), linear in the normalised
# profile, with the table G (radial class x axial
# lattice offset x time) learned by Adam from FDTD traces of random showers
# through the library's kernels (f32 master: sur_lattice_fwd_f32 / _bwd /
# sur_adam).  The weights served are bf16: the table split into a bf16 part
# and a bf16 remainder (sur_split_bf16), so that sums with cancellation keep
# nearly f32 precision.  Inference for a batch of profiles at one antenna is
# one tensor-core GEMM with split operands ([q_hi, q_hi, q_lo] times
# [W_hi; W_lo; W_hi], f32 accumulation) against the antenna's weight matrix.
# Antennas off the lattice, or outside its range, go to FDTD.

@dataclass
class LatticeGeometry:
    K: int = 128        # profile bins
    NR: int = 31        # radial classes
    m_lo: int = 3       # axial lattice index range of the antennas
    m_hi: int = 115
    T: int = 1024       # trace samples (every second step)
    S: int = 4          # samples between the passages of consecutive bins
    J: int = 4          # lead samples of a bin's response (one bin)

    @classmethod
    def of(cls, grid, ir, m, decim: int = 2):
        cells = int(round(grid.bin_dz / grid.dx))
        steps_per_bin = int(round(grid.bin_dz / (grid.v * grid.dt)))
        assert steps_per_bin % decim == 0
        return cls(K=grid.n_bins, NR=int(ir.max()) + 1, m_lo=int(m.min()), m_hi=int(m.max()),
                   T=grid.steps // decim, S=steps_per_bin // decim, J=steps_per_bin // decim)


class Lattice:
    """The learned bin-response table (f32 master, bf16 copy, gradient, Adam
    moments) on the current CUDA device."""

    def __init__(self, geo: LatticeGeometry, c_out: float = 1.0):
        import torch
        self.geo = geo
        self.c_out = float(c_out)
        self.t = 0
        shp = (geo.NR, self.D, geo.T)
        z = lambda dt=torch.float32: torch.zeros(shp, dtype=dt, device="cuda")
        self.G, self.dG, self.m, self.v = z(), z(), z(), z()
        self.Ghi, self.Glo = z(torch.bfloat16), z(torch.bfloat16)   # the bf16 weights served
        self._split = False
        self._ws = {}

    @property
    def D(self) -> int:
        # offsets m - k for m in [m_lo, m_hi], k in [0, K): index m - k + moff
        return self.geo.m_hi - self.geo.m_lo + self.geo.K

    @property
    def moff(self) -> int:
        return self.geo.K - 1 - self.geo.m_lo

    @property
    def n_params(self) -> int:
        return self.G.numel()

    def _w(self, B):
        import torch
        if B not in self._ws:
            e = lambda *sh: torch.empty(sh, dtype=torch.float32, device="cuda")
            self._ws = {B: {"qn": e(B, self.geo.K), "s": e(B), "y": e(B, self.geo.T), "tn": e(B, self.geo.T),
                            "dy": e(B, self.geo.T), "loss": e(1)}}
        return self._ws[B]

    def split(self):
        """The bf16 weights (part and remainder) from the f32 master."""
        check(sur_split_bf16(_p(self.G), _p(self.Ghi), _p(self.Glo), self.G.numel(), _stream()), "sur_split_bf16")
        self._split = True

    def _fwd(self, q, ant, scale_out, master=False):
        g = self.geo
        B = q.shape[0]
        w = self._w(B)
        st = _stream()
        check(sur_normalize_rows(_p(q), B, g.K, _p(w["qn"]), _p(w["s"]), st), "sur_normalize_rows")
        if master:
            check(sur_lattice_fwd_f32(_p(self.G), _p(w["qn"]), _p(ant), B, g.K, g.NR, self.D, g.T, g.S, g.J,
                                      self.moff, _p(w["y"]), st), "sur_lattice_fwd_f32")
        else:
            if not self._split:
                self.split()
            check(sur_lattice_fwd(_p(self.Ghi), _p(self.Glo), _p(w["qn"]), _p(ant), B, g.K, g.NR, self.D, g.T, g.S,
                                  g.J, self.moff, _p(w["y"]), st), "sur_lattice_fwd")
        if scale_out:
            check(sur_scale_rows(_p(w["y"]), B, g.T, _p(w["s"]), self.c_out, 0, st), "sur_scale_rows")
        return w["y"]

    def forward(self, q, ant):
        """Traces [B, T] for profiles q [B, K] (C per bin, f32) at antennas
        ant [B, 2] (int32: radial class, bin index), device tensors."""
        return self._fwd(q, ant, True)

    def train_batch(self, q, ant, trace, lr, b1=0.9, b2=0.999, eps=1e-8, relative=False):
        """One Adam step on the mean squared error of the traces, each divided
        by peak|q| c_out (relative=False) or by its own peak (relative=True:
        every trace's relative error weighs the same); returns the loss
        (device tensor)."""
        g = self.geo
        B = q.shape[0]
        w = self._w(B)
        st = _stream()
        self._fwd(q, ant, False, master=True)
        if relative:
            if "st" not in w:
                import torch
                w["st"] = torch.empty(B, dtype=torch.float32, device="cuda")
            check(sur_normalize_rows(_p(trace), B, g.T, _p(w["tn"]), _p(w["st"]), st), "sur_normalize_rows")
            # model trace / its target's peak = y_n c_out s_q / s_t
            check(sur_scale_rows(_p(w["y"]), B, g.T, _p(w["s"]), self.c_out, 0, st), "sur_scale_rows")
            check(sur_scale_rows(_p(w["y"]), B, g.T, _p(w["st"]), 1.0, 1, st), "sur_scale_rows")
        else:
            w["tn"].copy_(trace)
            check(sur_scale_rows(_p(w["tn"]), B, g.T, _p(w["s"]), 1.0 / self.c_out, 1, st), "sur_scale_rows")
        check(sur_mse(_p(w["y"]), _p(w["tn"]), B * g.T, _p(w["dy"]), _p(w["loss"]), st), "sur_mse")
        if relative:   # back to the gradient with respect to y_n
            check(sur_scale_rows(_p(w["dy"]), B, g.T, _p(w["s"]), self.c_out, 0, st), "sur_scale_rows")
            check(sur_scale_rows(_p(w["dy"]), B, g.T, _p(w["st"]), 1.0, 1, st), "sur_scale_rows")
        self.dG.zero_()
        check(sur_lattice_bwd(_p(w["dy"]), _p(w["qn"]), _p(ant), B, g.K, g.NR, self.D, g.T, g.S, g.J, self.moff,
                              _p(self.dG), st), "sur_lattice_bwd")
        self.t += 1
        check(sur_adam(_p(self.G), None, _p(self.dG), _p(self.m), _p(self.v), self.G.numel(), lr, b1, b2, eps, self.t,
                       st), "sur_adam")
        self._split = False
        return w["loss"]

    def predict(self, q, ant, chunk: int = 8192):
        import torch
        out = torch.empty(q.shape[0], self.geo.T, dtype=torch.float32, device="cuda")
        for lo in range(0, q.shape[0], chunk):
            hi = min(q.shape[0], lo + chunk)
            out[lo:hi].copy_(self.forward(q[lo:hi].contiguous(), ant[lo:hi].contiguous()))
        return out

    def predict_grid(self, q, ants):
        """Every profile q [P, K] at every antenna ants [A, 2]: traces
        [A, P, T]: one batched tensor-core GEMM (tcgen05: bf16 operands, f32
        accumulation in tensor memory) of the split profiles [hi, hi, lo]
        [P, 3K] with each antenna's K-major weights [W_hi; W_lo; W_hi]^T
        [T, 3K], both padded to a row of KP = 3K rounded up to 8, the profile
        scale applied in its epilogue."""
        import torch
        g = self.geo
        P, A, K = q.shape[0], ants.shape[0], self.geo.K
        KP = (3 * K + 7) // 8 * 8
        st = _stream()
        if not self._split:
            self.split()
        qn = torch.empty(P, K, dtype=torch.float32, device="cuda")
        s = torch.empty(P, dtype=torch.float32, device="cuda")
        check(sur_normalize_rows(_p(q), P, K, _p(qn), _p(s), st), "sur_normalize_rows")
        Q3 = torch.empty(P, KP, dtype=torch.bfloat16, device="cuda")
        check(sur_split3_bf16(_p(qn), P, K, _p(Q3), KP, st), "sur_split3_bf16")
        W3 = torch.zeros(A, g.T, KP, dtype=torch.bfloat16, device="cuda")
        for koff, tab in ((0, self.Ghi), (K, self.Glo), (2 * K, self.Ghi)):
            check(sur_lattice_weights_kmajor(_p(tab), _p(ants), A, K, g.NR, self.D, g.T, g.S, g.J, self.moff, _p(W3),
                                             KP, koff, st), "sur_lattice_weights_kmajor")
        out = torch.empty(A, P, g.T, dtype=torch.float32, device="cuda")
        # one launch for all antennas, the profile scale fused into the epilogue
        check(sur_gemm_bf16_batched(_p(Q3), KP, 0, _p(W3), KP, g.T * KP, _p(out), g.T, P * g.T, P, g.T, KP, A, _p(s),
                                    self.c_out, st), "sur_gemm_bf16_batched")
        return out


@dataclass
class LatticeData:
    q: object          # [R, K] f32 device: the profile of each FDTD run
    trace: object      # [R, A, T] f32 device: Ez at every lattice antenna, every `decim`-th step
    ant: object        # [A, 2] int32 device: (radial class, bin index) of each antenna
    fdtd_s: float = 0.0


def generate_lattice(grid, runs, ir, m, xyz, decim: int = 2, log=None) -> LatticeData:
    """One FDTD run of the library per shower of `runs` (workloads.surrogate_runs;
    their own detectors are ignored) on the lattice grid, recording Ez at every
    lattice antenna (one run gives them all, Sec. III.B)."""
    import torch
    steps, A = grid.steps, xyz.shape[0]
    T = steps // decim
    q_all = torch.empty(len(runs), grid.n_bins, dtype=torch.float32, device="cuda")
    tr_all = torch.empty(len(runs), A, T, dtype=torch.float32, device="cuda")
    lw = lateral_nkg(grid.lateral["L"], grid.dx, grid.lateral["r_moliere"], grid.lateral["age"],
                     grid.lateral["nsub"], grid.lateral["r_cut"])
    sim = Simulation(grid.nx, grid.ny, grid.nz, grid.dx, grid.dt, grid.eps_r, grid.boundary, grid.npml)
    sim.set_probes(xyz, steps)
    buf = torch.empty(A, steps, 2, dtype=torch.float32, device="cuda")
    t_fdtd = 0.0
    for r, run in enumerate(runs):
        q = profile_gaisser_hillas(grid.z0, grid.bin_dz, grid.n_bins, run["z1"], run["zmax"], run["lam"],
                                   run["nmax"], grid.profile["frac"])
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim.reset()
        sim.set_shower(q, grid.z0, grid.bin_dz, grid.v, lw, grid.lateral["L"])
        sim.step(steps)
        check(fdtd_probes(sim.h, _p(buf), 1), "fdtd_probes")
        torch.cuda.synchronize()
        t_fdtd += time.perf_counter() - t0
        tr_all[r].copy_(buf[:, decim - 1::decim, 0])
        q_all[r].copy_(torch.tensor(q, dtype=torch.float32))
        if log and (r + 1) % max(1, len(runs) // 5) == 0:
            log(f"fdtd run {r + 1}/{len(runs)}: {t_fdtd / (r + 1):.3f} s per run")
    sim.close()
    ant = torch.tensor(np.stack([ir, m], 1), dtype=torch.int32, device="cuda")
    return LatticeData(q_all, tr_all, ant, t_fdtd)


def train_lattice(data: LatticeData, geo: LatticeGeometry, steps: int, batch: int = 1024, lr: float = 3e-3,
                  seed: int = 0, log=None, relative: bool = False) -> Lattice:
    """Adam on random (shower, antenna) pairs of `data`; the learning rate
    decays by cosine to 1 % of `lr` (relative: see Lattice.train_batch)."""
    import torch
    R, A, _ = data.trace.shape
    s = data.q.abs().amax(dim=1)
    c_out = float(torch.sqrt(torch.mean((data.trace / s[:, None, None]) ** 2)).item())
    net = Lattice(geo, c_out=c_out)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    for it in range(steps):
        ri = torch.randint(0, R, (batch,), device="cuda", generator=gen)
        ai = torch.randint(0, A, (batch,), device="cuda", generator=gen)
        lr_t = lr * (0.01 + 0.99 * 0.5 * (1.0 + math.cos(math.pi * it / steps)))
        loss = net.train_batch(data.q[ri].contiguous(), data.ant[ai].contiguous(), data.trace[ri, ai].contiguous(),
                               lr_t, relative=relative)
        if log and it % max(1, steps // 10) == 0:
            log(f"lattice step {it} loss {float(loss.item()):.3e}")
    return net
