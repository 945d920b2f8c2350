"""Python binding of libfdtd_gb300.so (GB300 near-field FDTD of Askaryan pulses).

Argument marshalling only: every step of the field update, the source deposit,
the boundary and the detector readout runs in the library's CUDA kernels.  The
functions keep the C names of ``include/fdtd.h``; ``Simulation`` wraps a handle.
PyTorch is used for device buffers and streams only.  There is no CPU fallback:
importing this package fails if the compiled library is missing.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libfdtd_gb300.so")

FDTD_PEC, FDTD_MUR1, FDTD_CPML = 0, 1, 2
FDTD_OK = 0
STATUS = {0: "FDTD_OK", -1: "FDTD_ERR_ARG", -2: "FDTD_ERR_CFL", -3: "FDTD_ERR_OOM",
          -4: "FDTD_ERR_UNSTABLE", -5: "FDTD_ERR_CUDA", -6: "FDTD_ERR_TIMEOUT",
          -7: "FDTD_ERR_CAPACITY"}
COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -c 'import __graft_entry__ as g; g.build()'` (no CPU fallback exists)")

_d, _i, _vp, _sz = C.c_double, C.c_int, C.c_void_p, C.c_size_t
_pd, _pf, _pi = C.POINTER(C.c_double), C.POINTER(C.c_float), C.POINTER(C.c_int)
_pi64 = C.POINTER(C.c_int64)

lib = C.CDLL(LIB_PATH)
_SIGS = {
    "fdtd_create": (_i, [C.POINTER(_vp), _i, _i, _i, _d, _d, _d, _i, _i, _vp]),
    "fdtd_destroy": (None, [_vp]),
    "fdtd_set_shower": (_i, [_vp, _pd, _i, _d, _d, _i, _d, _pd, _i]),
    "fdtd_clear_shower": (_i, [_vp]),
    "fdtd_set_probes": (_i, [_vp, _pd, _i, _i]),
    "fdtd_probe_nodes": (_i, [_vp, _pi]),
    "fdtd_step": (_i, [_vp, _i]),
    "fdtd_sync": (_i, [_vp]),
    "fdtd_steps_done": (_i, [_vp, _pi64]),
    "fdtd_probes": (_i, [_vp, _vp, _i]),
    "fdtd_fields": (_i, [_vp, _i, _vp, _i]),
    "fdtd_set_field": (_i, [_vp, _i, _vp, _i]),
    "fdtd_reset": (_i, [_vp]),
    "fdtd_energy": (_i, [_vp, _pd]),
    "fdtd_energy_noalloc": (_i, [_vp, _i, _i, _i, _d, _d, _i, _vp, _pd]),
    "fdtd_adjoint_step": (_i, [_vp, _i]),
    "fdtd_adjoint_gradient": (_i, [_vp, _vp, _i, _vp, _i]),
    "fdtd_save_state": (_i, [_vp, _vp, C.POINTER(_sz)]),
    "fdtd_load_state": (_i, [_vp, _vp, _sz]),
    "fdtd_timing_begin": (_i, [_vp, _i]),
    "fdtd_timing_end": (_i, [_vp, _pd, _pi]),
    "fdtd_launch_count": (_i, [_vp, _pi64]),
    "fdtd_timed_cells": (_i, [_vp, _pi64]),
    "fdtd_kernel_name": (C.c_char_p, [_vp]),
    "fdtd_set_kernel": (_i, [_vp, _i]),
    "fdtd_set_watchdog": (_i, [_vp, _i]),
    "fdtd_strerror": (C.c_char_p, [_i]),
    "fdtd_profile_gaussian": (_i, [_d, _d, _i, _d, _d, _d, _pd]),
    "fdtd_profile_greisen": (_i, [_d, _i, _d, _d, _d, _d, _pd]),
    "fdtd_profile_gaisser_hillas": (_i, [_d, _d, _i, _i, _pd, _pd, _pd, _pd, _d, _pd]),
    "fdtd_lateral_gaussian": (_i, [_i, _d, _pd]),
    "fdtd_lateral_nkg": (_i, [_i, _d, _d, _d, _i, _d, _pd]),
    "cyl_rings_gaussian": (_i, [_i, _d, _d, _pd]),
    # learned surrogate kernels (surrogate.h); pointers are device addresses
    "sur_gemm_bf16": (_i, [_vp, _i, _i, _vp, _i, _i, _vp, _i, _vp, _i, _i, _i, _vp, _i, _i, _vp]),
    "sur_gemm_set_path": (_i, [_i]),
    "sur_gemm_tc_launches": (C.c_longlong, []),
    "sur_gemm_tc_failed": (_i, []),
    "sur_gemm_bf16_batched": (_i, [_vp, _i, C.c_longlong, _vp, _i, C.c_longlong, _vp, _i, C.c_longlong, _i, _i, _i,
                                   _i, _vp, C.c_float, _vp]),
    "sur_conv1d_fwd": (_i, [_vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "sur_conv1d_bwd": (_i, [_vp, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _vp]),
    "sur_relu_bwd": (_i, [_vp, _vp, _vp, _vp, C.c_longlong, _vp]),
    "sur_bias_grad": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "sur_cast_bf16": (_i, [_vp, _vp, C.c_longlong, _vp]),
    "sur_concat_bf16": (_i, [_vp, _i, _vp, _i, _vp, _i, _vp]),
    "sur_mse": (_i, [_vp, _vp, C.c_longlong, _vp, _vp, _vp]),
    "sur_adam": (_i, [_vp, _vp, _vp, _vp, _vp, C.c_longlong, C.c_float, C.c_float, C.c_float, C.c_float, _i, _vp]),
    "sur_normalize_rows": (_i, [_vp, _i, _i, _vp, _vp, _vp]),
    "sur_antenna_features": (_i, [_vp, _i, C.c_float, C.c_float, C.c_float, C.c_float, _vp, _vp]),
    "sur_scale_rows": (_i, [_vp, _i, _i, _vp, C.c_float, _i, _vp]),
    "sur_pairs": (_i, [_vp, _i, _i, C.c_float, C.c_float, _vp, _vp]),
    "sur_assemble": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, C.c_float, C.c_float, C.c_float, _i, _vp, _vp]),
    "sur_assemble_bwd": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, C.c_float, C.c_float, C.c_float, _i, _vp, _vp,
                              _vp]),
    "sur_lattice_fwd": (_i, [_vp, _vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp, _vp]),
    "sur_lattice_fwd_f32": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp, _vp]),
    "sur_split_bf16": (_i, [_vp, _vp, _vp, C.c_longlong, _vp]),
    "sur_lattice_bwd": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp, _vp]),
    "sur_lattice_weights": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp, _vp]),
    "sur_lattice_weights_kmajor": (_i, [_vp, _vp, _i, _i, _i, _i, _i, _i, _i, _i, _vp, _i, _i, _vp]),
    "sur_split3_bf16": (_i, [_vp, _i, _i, _vp, _i, _vp]),
    # batched persistent stepping (batch.h)
    "fdtd_batch_create": (_i, [C.POINTER(_vp), C.POINTER(_vp), _i]),
    "fdtd_batch_destroy": (None, [_vp]),
    "fdtd_batch_step": (_i, [_vp, _i]),
    "fdtd_batch_sync": (_i, [_vp]),
    "fdtd_batch_set_config": (_i, [_vp, _i, _i]),
    "fdtd_batch_get_config": (_i, [_vp, _pi, _pi]),
    "fdtd_batch_tune": (_i, [_vp, _i, _pi]),
    "fdtd_batch_graph_mode": (_i, [_vp]),
    "fdtd_batch_set_solo": (_i, [_vp, C.c_longlong]),
    "fdtd_batch_get_solo": (_i, [_vp, C.POINTER(C.c_longlong), _pi]),
    "fdtd_batch_set_wait_limit": (_i, [_vp, C.c_longlong]),
    # 2D axisymmetric solver (cyl.h)
    "cyl_create": (_i, [C.POINTER(_vp), _i, _i, _d, _d, _d, _i, _vp]),
    "cyl_destroy": (None, [_vp]),
    "cyl_set_shower": (_i, [_vp, _pd, _i, _d, _d, _d, _pd, _i]),
    "cyl_set_probes": (_i, [_vp, _pd, _i, _i]),
    "cyl_step": (_i, [_vp, _i]),
    "cyl_set_kernel": (_i, [_vp, _i, _i]),
    "cyl_tune": (_i, [_vp, _i, _pi]),
    "cyl_kernel_info": (_i, [_vp, _pi, _pi, _pi]),
    "cyl_kernel_name": (C.c_char_p, [_vp]),
    "cyl_steps_done": (_i, [_vp, _pi64]),
    "cyl_sync": (_i, [_vp]),
    "cyl_probes": (_i, [_vp, _vp, _i]),
    "cyl_fields": (_i, [_vp, _i, _vp, _i]),
    "cyl_set_field": (_i, [_vp, _i, _vp, _i]),
    "cyl_reset": (_i, [_vp]),
    "cyl_launch_count": (_i, [_vp, _pi64]),
    # spectra of detector traces (spectra.h)
    "fdtd_trace_spectrum": (_i, [_vp, _i, _i, _i, _pd, _pi, _d, _d, _d, _pd, _i, _vp, _i, _vp]),
    "fdtd_theta_coef": (_i, [_pd, _i, _pd]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args
    globals()[_name] = _f


class FdtdError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)} ({fdtd_strerror(code).decode()})")


def check(code: int, where: str = "fdtd") -> int:
    if code != FDTD_OK:
        raise FdtdError(code, where)
    return code


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_pd)


# ---- shower tables ---------------------------------------------------------

def profile_gaussian(z0, bin_dz, n_bins, z_peak, l, q_max):
    out = np.zeros(n_bins)
    check(fdtd_profile_gaussian(z0, bin_dz, n_bins, z_peak, l, q_max, _dp(out)), "profile_gaussian")
    return out


def profile_greisen(bin_dz, n_bins, E0, Ec, X0, frac):
    out = np.zeros(n_bins)
    check(fdtd_profile_greisen(bin_dz, n_bins, E0, Ec, X0, frac, _dp(out)), "profile_greisen")
    return out


def profile_gaisser_hillas(z0, bin_dz, n_bins, z1, zmax, lam, nmax, frac):
    a = [np.ascontiguousarray(x, dtype=np.float64) for x in (z1, zmax, lam, nmax)]
    out = np.zeros(n_bins)
    check(fdtd_profile_gaisser_hillas(z0, bin_dz, n_bins, a[0].size, *[_dp(x) for x in a], frac,
                                      _dp(out)), "profile_gaisser_hillas")
    return out


def lateral_gaussian(L, sigma_cells):
    out = np.zeros((2 * L + 1) ** 2)
    check(fdtd_lateral_gaussian(L, sigma_cells, _dp(out)), "lateral_gaussian")
    return out


def lateral_nkg(L, dx, r_moliere, age, nsub, r_cut):
    out = np.zeros((2 * L + 1) ** 2)
    check(fdtd_lateral_nkg(L, dx, r_moliere, age, nsub, r_cut, _dp(out)), "lateral_nkg")
    return out


def tables(w):
    """Profile and lateral tables of a ``workloads.Workload`` from the library's
    own host generators."""
    p, lt = w.profile, w.lateral
    if p["kind"] == "gaussian":
        q = profile_gaussian(w.z0, w.bin_dz, w.n_bins, p["z_peak"], p["l"], p["q_max"])
    elif p["kind"] == "greisen":
        q = profile_greisen(w.bin_dz, w.n_bins, p["E0_eV"], p["Ec_eV"], p["X0_m"], p["frac"])
    elif p["kind"] == "gh":
        q = profile_gaisser_hillas(w.z0, w.bin_dz, w.n_bins, p["z1"], p["zmax"], p["lam"],
                                   p["nmax"], p["frac"])
    elif p["kind"] == "table":
        q = np.asarray(p["q"], dtype=np.float64)
    else:
        raise ValueError(p["kind"])
    if lt["kind"] == "gaussian":
        lw = lateral_gaussian(lt["L"], lt["sigma_cells"])
    elif lt["kind"] == "nkg":
        lw = lateral_nkg(lt["L"], w.dx, lt["r_moliere"], lt["age"], lt["nsub"], lt["r_cut"])
    elif lt["kind"] == "table":
        lw = np.asarray(lt["w"], dtype=np.float64)
    else:
        raise ValueError(lt["kind"])
    return q, lw


def cyl_tables(w):
    """Charge table and ring weights of a ``workloads.CylWorkload`` (the
    paper's Gaussian shower model, Sec. III.B) from the library's own host
    generators."""
    s = w.shower
    if s["kind"] != "gaussian":
        raise ValueError(s["kind"])
    q = profile_gaussian(w.z0, w.bin_dz, s["n_bins"], s["z_peak"], s["l"], s["q_max"])
    rings = np.zeros(s["n_rings"])
    check(cyl_rings_gaussian(s["n_rings"], w.d, s["sigma_r"], _dp(rings)), "cyl_rings_gaussian")
    return q, rings


# ---- simulation handle -------------------------------------------------------

class Simulation:
    """One simulation on the current CUDA device.  ``stream`` is a
    ``torch.cuda.Stream`` (or a raw cudaStream_t int); default: torch's current
    stream."""

    def __init__(self, nx, ny, nz, dx, dt, eps_r, boundary=FDTD_MUR1, npml=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        raw = stream if isinstance(stream, int) else stream.cuda_stream
        h = _vp()
        check(fdtd_create(C.byref(h), nx, ny, nz, dx, dt, eps_r, boundary, npml, _vp(raw)),
              "fdtd_create")
        self.h = h
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dt, self.eps_r = dx, dt, eps_r
        self.boundary, self.npml = boundary, npml
        self.np, self.max_steps = 0, 0

    @classmethod
    def from_workload(cls, w, max_steps: Optional[int] = None, stream=None, kernel=None):
        s = cls(w.nx, w.ny, w.nz, w.dx, w.dt, w.eps_r, w.boundary, w.npml, stream=stream)
        if kernel is not None:
            s.set_kernel(kernel)
        q, lw = tables(w)
        s.set_shower(q, w.z0, w.bin_dz, w.v, lw, w.lateral["L"])
        s.set_probes(w.probes_xyz, w.steps if max_steps is None else max_steps)
        return s

    def close(self):
        if getattr(self, "h", None):
            fdtd_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    def set_shower(self, q, z0, bin_dz, v, w, L, axis=2):
        q = np.ascontiguousarray(q, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        check(fdtd_set_shower(self.h, _dp(q), q.size, z0, bin_dz, axis, v, _dp(w), L), "fdtd_set_shower")
        self.n_bins = q.size

    def clear_shower(self):
        check(fdtd_clear_shower(self.h), "fdtd_clear_shower")

    def set_probes(self, xyz, max_steps):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        check(fdtd_set_probes(self.h, _dp(xyz), xyz.shape[0], max_steps), "fdtd_set_probes")
        self.np, self.max_steps = xyz.shape[0], max_steps

    def probe_nodes(self):
        out = np.zeros((self.np, 3), dtype=np.int32)
        check(fdtd_probe_nodes(self.h, out.ctypes.data_as(_pi)), "fdtd_probe_nodes")
        return out

    def step(self, n=1):
        check(fdtd_step(self.h, n), "fdtd_step")

    def sync(self):
        check(fdtd_sync(self.h), "fdtd_sync")

    @property
    def steps_done(self):
        v = C.c_int64()
        check(fdtd_steps_done(self.h, C.byref(v)), "fdtd_steps_done")
        return v.value

    def probes(self, out=None):
        """Traces [n_probes][max_steps][2] (Ez, E_r): numpy, or into a CUDA tensor."""
        if out is not None:
            check(fdtd_probes(self.h, _vp(out.data_ptr()), 1), "fdtd_probes")
            return out
        a = np.zeros((self.np, self.max_steps, 2), dtype=np.float32)
        check(fdtd_probes(self.h, _vp(a.ctypes.data), 0), "fdtd_probes")
        return a

    def spectrum(self, freqs, theta=None, coef=None, gate=None, taper=0.0):
        """E_omega of every detector's trace (trace_spectrum; sample s at (s + 1) dt).
        theta: per-detector polar angles for the theta-hat component; else coef
        (default: E_z).  Returns a complex64 CUDA tensor [n_probes, n_freq]."""
        import torch
        tr = torch.empty((self.np, self.max_steps, 2), dtype=torch.float32, device="cuda")
        self.probes(out=tr)
        if theta is not None:
            coef = theta_coef(theta)
        return trace_spectrum(tr, self.dt, freqs, t0=self.dt, coef=coef, gate=gate, taper=taper,
                              stream=self.stream)

    def field(self, comp, out=None):
        c = COMPONENTS.index(comp) if isinstance(comp, str) else comp
        if out is not None:
            check(fdtd_fields(self.h, c, _vp(out.data_ptr()), 1), "fdtd_fields")
            return out
        a = np.zeros(self.shape, dtype=np.float32)
        check(fdtd_fields(self.h, c, _vp(a.ctypes.data), 0), "fdtd_fields")
        return a

    def set_field(self, comp, arr):
        c = COMPONENTS.index(comp) if isinstance(comp, str) else comp
        a = np.ascontiguousarray(arr, dtype=np.float32)
        assert a.shape == self.shape
        check(fdtd_set_field(self.h, c, _vp(a.ctypes.data), 0), "fdtd_set_field")

    def reset(self):
        check(fdtd_reset(self.h), "fdtd_reset")

    def energy(self):
        e = C.c_double()
        check(fdtd_energy(self.h, C.byref(e)), "fdtd_energy")
        return e.value

    def save_state(self) -> bytes:
        n = _sz(0)
        check(fdtd_save_state(self.h, None, C.byref(n)), "fdtd_save_state")
        buf = C.create_string_buffer(n.value)
        check(fdtd_save_state(self.h, C.cast(buf, _vp), C.byref(n)), "fdtd_save_state")
        return buf.raw

    def load_state(self, blob: bytes):
        buf = C.create_string_buffer(blob, len(blob))
        check(fdtd_load_state(self.h, C.cast(buf, _vp), len(blob)), "fdtd_load_state")

    def timing_begin(self, max_launches):
        check(fdtd_timing_begin(self.h, max_launches), "fdtd_timing_begin")

    def timing_end(self):
        ms, n = C.c_double(), C.c_int()
        check(fdtd_timing_end(self.h, C.byref(ms), C.byref(n)), "fdtd_timing_end")
        return ms.value, n.value

    @property
    def launches(self):
        v = C.c_int64()
        check(fdtd_launch_count(self.h, C.byref(v)), "fdtd_launch_count")
        return v.value

    @property
    def timed_cells(self):
        """Cells one launch of the timed kernel updates."""
        v = C.c_int64()
        check(fdtd_timed_cells(self.h, C.byref(v)), "fdtd_timed_cells")
        return v.value

    @property
    def kernel_name(self):
        return fdtd_kernel_name(self.h).decode()

    def set_kernel(self, which: int):
        """2: two steps per pass (default on PEC and CPML grids from 3 * 2^22 cells),
        1: one-pass tile z-march (default otherwise), 0: unfused H sweep then E sweep."""
        check(fdtd_set_kernel(self.h, which), "fdtd_set_kernel")

    def adjoint_step(self, n=1):
        """n transposed steps of the fields and CPML memory."""
        check(fdtd_adjoint_step(self.h, n), "fdtd_adjoint_step")

    def adjoint_gradient(self, dl_dtrace, n_steps, out=None):
        """dL/dq of the charge table from dL/d(trace), a contiguous float32
        CUDA tensor [n_probes][max_steps][2]; numpy float64, or into a float64
        CUDA tensor.  Leaves the handle reset."""
        import torch
        if (dl_dtrace.dtype != torch.float32 or not dl_dtrace.is_cuda or not dl_dtrace.is_contiguous()
                or tuple(dl_dtrace.shape) != (self.np, self.max_steps, 2)):
            raise ValueError(f"dl_dtrace: need a contiguous float32 CUDA tensor [{self.np}, {self.max_steps}, 2]")
        if out is not None:
            check(fdtd_adjoint_gradient(self.h, _vp(dl_dtrace.data_ptr()), n_steps, _vp(out.data_ptr()), 1),
                  "fdtd_adjoint_gradient")
            return out
        g = np.zeros(self.n_bins, dtype=np.float64)
        check(fdtd_adjoint_gradient(self.h, _vp(dl_dtrace.data_ptr()), n_steps, _vp(g.ctypes.data), 0),
              "fdtd_adjoint_gradient")
        return g


# ---- 2D axisymmetric solver ---------------------------------------------------

CYL_COMPONENTS = ("Er", "Ez", "Hphi")


def trace_spectrum(traces, dt, freqs, t0=0.0, coef=None, gate=None, taper=0.0, stream=None):
    """E_omega of detector traces (spectra.h), Sec. V: dt sum_m g_m x_{first+m}
    exp(i 2 pi f t_{first+m}), t_n = t0 + n dt, x_n = sum_c coef_c X[n][c].

    traces: float32 CUDA tensor [n_traces, n_t, n_comp] (or [n_traces, n_t]);
    coef: [n_traces, n_comp] (default: the first component); gate: [n_traces, 2]
    (first, count) (default: the whole trace); taper: Tukey fraction.
    Returns a complex64 CUDA tensor [n_traces, n_freq] (asynchronous on the stream)."""
    import torch
    if not (isinstance(traces, torch.Tensor) and traces.is_cuda and traces.dtype == torch.float32):
        raise ValueError("traces: need a float32 CUDA tensor")
    t = (traces if traces.dim() == 3 else traces.unsqueeze(-1)).contiguous()
    n_tr, n_t, n_c = t.shape
    f = np.ascontiguousarray(np.asarray(freqs, dtype=np.float64).ravel())
    co = None if coef is None else np.ascontiguousarray(np.asarray(coef, dtype=np.float64).reshape(n_tr, n_c))
    ga = None if gate is None else np.ascontiguousarray(np.asarray(gate, dtype=np.int32).reshape(n_tr, 2))
    if stream is None:
        stream = torch.cuda.current_stream(t.device)
    raw = stream if isinstance(stream, int) else stream.cuda_stream
    out = torch.empty((n_tr, f.size, 2), dtype=torch.float32, device=t.device)
    check(fdtd_trace_spectrum(_vp(t.data_ptr()), n_tr, n_t, n_c, None if co is None else _dp(co),
                              None if ga is None else ga.ctypes.data_as(_pi), float(taper), float(dt), float(t0),
                              _dp(f), f.size, _vp(out.data_ptr()), 1, _vp(raw)), "fdtd_trace_spectrum")
    return torch.view_as_complex(out)


def theta_coef(theta):
    """(E_z, E_r) weights of the theta-hat component (fdtd_theta_coef)."""
    th = np.ascontiguousarray(np.asarray(theta, dtype=np.float64).ravel())
    out = np.zeros((th.size, 2))
    check(fdtd_theta_coef(_dp(th), th.size, _dp(out)), "fdtd_theta_coef")
    return out


class Cylinder:
    """The paper's (E_r, E_z, H_phi) solver on an (r, z) grid of nr x nz cells
    (cyl.h).  ``stream``: a ``torch.cuda.Stream`` or raw cudaStream_t int;
    default: torch's current stream."""

    def __init__(self, nr, nz, d, dt, eps_r, boundary=FDTD_MUR1, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = stream
        raw = stream if isinstance(stream, int) else stream.cuda_stream
        h = _vp()
        check(cyl_create(C.byref(h), nr, nz, d, dt, eps_r, boundary, _vp(raw)), "cyl_create")
        self.h = h
        self.nr, self.nz, self.d, self.dt, self.eps_r, self.boundary = nr, nz, d, dt, eps_r, boundary
        self.np, self.max_steps = 0, 0

    def close(self):
        if getattr(self, "h", None):
            cyl_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def shape(self, comp):
        c = CYL_COMPONENTS.index(comp) if isinstance(comp, str) else comp
        return ((self.nr, self.nz + 1), (self.nr + 1, self.nz), (self.nr, self.nz))[c]

    def set_shower(self, q, z0, bin_dz, v, w):
        q = np.ascontiguousarray(q, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        check(cyl_set_shower(self.h, _dp(q), q.size, z0, bin_dz, v, _dp(w), w.size), "cyl_set_shower")

    def set_probes(self, rz, max_steps):
        rz = np.ascontiguousarray(np.asarray(rz, dtype=np.float64).reshape(-1, 2))
        check(cyl_set_probes(self.h, _dp(rz), rz.shape[0], max_steps), "cyl_set_probes")
        self.np, self.max_steps = rz.shape[0], max_steps

    def set_kernel(self, which: int, seg_rows: int = 0):
        """0: two kernels per step; 1..5: wavefront variants (cyl.h), K steps per launch."""
        check(cyl_set_kernel(self.h, which, seg_rows), "cyl_set_kernel")

    def tune(self, launches: int = 2) -> int:
        """Segment length of the wavefront kernel by timing real steps (cyl_tune); returns the steps used."""
        used = C.c_int()
        check(cyl_tune(self.h, launches, C.byref(used)), "cyl_tune")
        return used.value

    @property
    def kernel_info(self):
        w, k, l = C.c_int(), C.c_int(), C.c_int()
        check(cyl_kernel_info(self.h, C.byref(w), C.byref(k), C.byref(l)), "cyl_kernel_info")
        return {"kernel": w.value, "kernel_name": cyl_kernel_name(self.h).decode(),
                "steps_per_launch": k.value, "seg_rows": l.value}

    def step(self, n=1):
        check(cyl_step(self.h, n), "cyl_step")

    def sync(self):
        check(cyl_sync(self.h), "cyl_sync")

    @property
    def steps_done(self):
        v = C.c_int64()
        check(cyl_steps_done(self.h, C.byref(v)), "cyl_steps_done")
        return v.value

    @property
    def launches(self):
        v = C.c_int64()
        check(cyl_launch_count(self.h, C.byref(v)), "cyl_launch_count")
        return v.value

    def probes(self, out=None):
        """Traces [n_probes][max_steps][2] (E_z, E_r): numpy, or into a CUDA tensor."""
        if out is not None:
            check(cyl_probes(self.h, _vp(out.data_ptr()), 1), "cyl_probes")
            return out
        a = np.zeros((self.np, self.max_steps, 2), dtype=np.float32)
        check(cyl_probes(self.h, _vp(a.ctypes.data), 0), "cyl_probes")
        return a

    def spectrum(self, freqs, theta=None, coef=None, gate=None, taper=0.0):
        """E_omega of every detector's trace (trace_spectrum; sample s at (s + 1) dt).
        theta: per-detector polar angles for the theta-hat component; else coef
        (default: E_z).  Returns a complex64 CUDA tensor [n_probes, n_freq]."""
        import torch
        tr = torch.empty((self.np, self.max_steps, 2), dtype=torch.float32, device="cuda")
        self.probes(out=tr)
        if theta is not None:
            coef = theta_coef(theta)
        return trace_spectrum(tr, self.dt, freqs, t0=self.dt, coef=coef, gate=gate, taper=taper,
                              stream=self.stream)

    def field(self, comp, out=None):
        c = CYL_COMPONENTS.index(comp) if isinstance(comp, str) else comp
        if out is not None:
            check(cyl_fields(self.h, c, _vp(out.data_ptr()), 1), "cyl_fields")
            return out
        a = np.zeros(self.shape(c), dtype=np.float32)
        check(cyl_fields(self.h, c, _vp(a.ctypes.data), 0), "cyl_fields")
        return a

    def set_field(self, comp, arr):
        """From a host array, or from a contiguous float32 CUDA tensor."""
        c = CYL_COMPONENTS.index(comp) if isinstance(comp, str) else comp
        if hasattr(arr, "data_ptr") and getattr(arr, "is_cuda", False):
            import torch
            if arr.dtype != torch.float32 or not arr.is_contiguous() or tuple(arr.shape) != self.shape(c):
                raise ValueError(f"{CYL_COMPONENTS[c]}: need a contiguous float32 tensor of shape {self.shape(c)}")
            check(cyl_set_field(self.h, c, _vp(arr.data_ptr()), 1), "cyl_set_field")
            return
        a = np.ascontiguousarray(arr, dtype=np.float32)
        if a.shape != self.shape(c):
            raise ValueError(f"{CYL_COMPONENTS[c]}: shape {a.shape}, expected {self.shape(c)}")
        check(cyl_set_field(self.h, c, _vp(a.ctypes.data), 0), "cyl_set_field")

    def reset(self):
        check(cyl_reset(self.h), "cyl_reset")


# ---- batched persistent stepping ------------------------------------------------

class Batch:
    """Several ``Simulation`` objects advanced together by one persistent
    kernel per launch (batch.h).  The simulations must outlive the batch."""

    def __init__(self, sims):
        self.sims = list(sims)
        arr = (_vp * len(self.sims))(*[s.h for s in self.sims])
        h = _vp()
        check(fdtd_batch_create(C.byref(h), arr, len(self.sims)), "fdtd_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            fdtd_batch_destroy(self.h)
            self.h = None

    __del__ = close

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def step(self, n=1):
        check(fdtd_batch_step(self.h, n), "fdtd_batch_step")

    def sync(self):
        check(fdtd_batch_sync(self.h), "fdtd_batch_sync")

    def set_config(self, chunk_planes=256, steps_per_launch=8):
        """z planes per chunk of the persistent kernel's tile items, steps per launch."""
        check(fdtd_batch_set_config(self.h, chunk_planes, steps_per_launch), "fdtd_batch_set_config")

    @property
    def config(self):
        c, s = C.c_int(), C.c_int()
        check(fdtd_batch_get_config(self.h, C.byref(c), C.byref(s)), "fdtd_batch_get_config")
        return {"chunk_planes": c.value, "steps_per_launch": s.value}

    def set_solo(self, min_cells=-1):
        """Simulations of at least min_cells cells step alone with their own
        selected path (-1: all share the persistent kernel)."""
        check(fdtd_batch_set_solo(self.h, int(min_cells)), "fdtd_batch_set_solo")

    @property
    def solo(self):
        m, k = C.c_longlong(), C.c_int()
        check(fdtd_batch_get_solo(self.h, C.byref(m), C.byref(k)), "fdtd_batch_get_solo")
        return {"min_cells": m.value, "n_solo": k.value}

    def tune(self, trial_steps=4):
        """Autotune on the batch itself; returns the steps the trials advanced."""
        used = C.c_int()
        check(fdtd_batch_tune(self.h, trial_steps, C.byref(used)), "fdtd_batch_tune")
        return used.value

    def set_wait_limit(self, cycles=0):
        """Bound of every grid-barrier wait in SM clock cycles (0: default)."""
        check(fdtd_batch_set_wait_limit(self.h, int(cycles)), "fdtd_batch_set_wait_limit")

    @property
    def graph_mode(self):
        return fdtd_batch_graph_mode(self.h)

