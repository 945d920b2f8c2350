"""FP64 CPU oracle of the 3D Yee FDTD near-field path (ctypes wrapper).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA library never imports it and shares no code with it.

The arithmetic lives in ``fdtd_oracle.c`` (plain C, FP64, ``-ffp-contract=off``);
each routine there cites the passage of the paper it restates.  This module only
marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fdtd_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")

PEC, MUR1, CPML = 0, 1, 2
COMPONENTS = ("Ex", "Ey", "Ez", "Hx", "Hy", "Hz")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, FP64, no FMA contraction)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-std=c11", "-D_DEFAULT_SOURCE", "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB)
        d, i, p, vp = C.c_double, C.c_int, C.POINTER(C.c_double), C.c_void_p
        L.orc_create.restype = vp
        L.orc_create.argtypes = [i, i, i, d, d, d, i, i]
        L.orc_destroy.argtypes = [vp]
        L.orc_set_shower.argtypes = [vp, p, i, d, d, d, p, i]
        L.orc_set_probes.argtypes = [vp, p, i, i]
        L.orc_step.argtypes = [vp, i]
        L.orc_steps_done.argtypes = [vp]
        L.orc_steps_done.restype = C.c_long
        L.orc_get_field.argtypes = [vp, i, p]
        L.orc_set_field.argtypes = [vp, i, p]
        L.orc_get_probes.argtypes = [vp, p]
        L.orc_get_probe_nodes.argtypes = [vp, C.POINTER(C.c_int)]
        L.orc_set_threads.argtypes = [i]
        L.orc_set_threads.restype = i
        L.orc_source_count.argtypes = [vp]
        L.orc_get_source.argtypes = [vp, C.POINTER(C.c_int64), p]
        for f in ("orc_kE", "orc_kH", "orc_eps"):
            getattr(L, f).argtypes = [vp]
            getattr(L, f).restype = d
        for f in ("orc_c0", "orc_mu0", "orc_eps0"):
            getattr(L, f).argtypes = []
            getattr(L, f).restype = d
        L.orc_profile_at.argtypes = [vp, d]
        L.orc_profile_at.restype = d
        L.orc_cpml_coefs.argtypes = [vp, i, p, p, p, p]
        L.orc_profile_gaussian.argtypes = [d, d, i, d, d, d, p]
        L.orc_greisen.argtypes = [d, d, d]
        L.orc_greisen.restype = d
        L.orc_profile_greisen.argtypes = [d, d, i, d, d, d, d, p]
        L.orc_profile_gh.argtypes = [d, d, i, i, p, p, p, p, d, p]
        L.orc_lateral_gaussian.argtypes = [i, d, p]
        L.orc_lateral_nkg.argtypes = [i, d, d, d, i, d, p]
        _lib = L
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def c0() -> float:
    return lib().orc_c0()


def mu0() -> float:
    return lib().orc_mu0()


def eps0() -> float:
    return lib().orc_eps0()


class Oracle:
    """One FP64 simulation.  Fields come back as (nz+1, ny+1, nx+1) arrays."""

    def __init__(self, nx, ny, nz, dx, dt, eps_r, boundary=MUR1, npml=0):
        self.L = lib()
        self.h = self.L.orc_create(nx, ny, nz, dx, dt, eps_r, boundary, npml)
        if not self.h:
            raise ValueError("oracle: bad grid / boundary arguments or out of memory")
        self.nx, self.ny, self.nz = nx, ny, nz
        self.dx, self.dt, self.eps_r = dx, dt, eps_r
        self.boundary, self.npml = boundary, (npml if boundary == CPML else 0)
        self.np = 0
        self.max_steps = 0

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.L.orc_destroy(h)
            self.h = None

    @property
    def shape(self):
        return (self.nz + 1, self.ny + 1, self.nx + 1)

    @property
    def kE(self):
        return self.L.orc_kE(self.h)

    @property
    def kH(self):
        return self.L.orc_kH(self.h)

    @property
    def eps(self):
        return self.L.orc_eps(self.h)

    def set_shower(self, q, z0, bin_dz, v, w, L):
        q = np.ascontiguousarray(q, dtype=np.float64)
        w = np.ascontiguousarray(w, dtype=np.float64)
        assert w.size == (2 * L + 1) ** 2
        rc = self.L.orc_set_shower(self.h, _dp(q), q.size, z0, bin_dz, v, _dp(w), L)
        if rc != 0:
            raise ValueError(f"oracle set_shower failed ({rc})")

    def set_probes(self, xyz, max_steps):
        xyz = np.ascontiguousarray(np.asarray(xyz, dtype=np.float64).reshape(-1, 3))
        rc = self.L.orc_set_probes(self.h, _dp(xyz), xyz.shape[0], max_steps)
        if rc != 0:
            raise ValueError(f"oracle set_probes failed ({rc})")
        self.np, self.max_steps = xyz.shape[0], max_steps

    def step(self, n=1):
        if self.L.orc_step(self.h, n) != 0:
            raise ValueError("oracle step failed")

    @property
    def steps_done(self):
        return self.L.orc_steps_done(self.h)

    def field(self, comp):
        c = COMPONENTS.index(comp) if isinstance(comp, str) else comp
        out = np.empty(self.shape, dtype=np.float64)
        self.L.orc_get_field(self.h, c, _dp(out))
        return out

    def set_field(self, comp, arr):
        c = COMPONENTS.index(comp) if isinstance(comp, str) else comp
        a = np.ascontiguousarray(arr, dtype=np.float64)
        assert a.shape == self.shape
        self.L.orc_set_field(self.h, c, _dp(a))

    def probes(self):
        out = np.zeros((self.np, self.max_steps, 2), dtype=np.float64)
        if self.np:
            self.L.orc_get_probes(self.h, _dp(out))
        return out

    def probe_nodes(self):
        out = np.zeros((self.np, 3), dtype=np.int32)
        if self.np:
            self.L.orc_get_probe_nodes(self.h, out.ctypes.data_as(C.POINTER(C.c_int)))
        return out

    def source(self):
        """J_z entries injected by the last step: (flat node index, value A/m^2)."""
        n = self.L.orc_source_count(self.h)
        idx = np.zeros(n, dtype=np.int64)
        val = np.zeros(n, dtype=np.float64)
        if n:
            self.L.orc_get_source(self.h, idx.ctypes.data_as(C.POINTER(C.c_int64)), _dp(val))
        return idx, val

    def profile_at(self, z):
        return self.L.orc_profile_at(self.h, z)

    def cpml_coefs(self, axis):
        n = (self.nx, self.ny, self.nz)[axis] + 1
        arrs = [np.zeros(n) for _ in range(4)]
        self.L.orc_cpml_coefs(self.h, axis, *[_dp(a) for a in arrs])
        return arrs  # aE, bE, aH, bH


# ---- shower tables (Sec. III.B) -------------------------------------------

def profile_gaussian(z0, bin_dz, nbins, z_peak, l, q_max):
    out = np.zeros(nbins)
    lib().orc_profile_gaussian(z0, bin_dz, nbins, z_peak, l, q_max, _dp(out))
    return out


def greisen(t, E0, Ec):
    return lib().orc_greisen(t, E0, Ec)


def profile_greisen(z0, bin_dz, nbins, E0, Ec, X0, frac):
    out = np.zeros(nbins)
    lib().orc_profile_greisen(z0, bin_dz, nbins, E0, Ec, X0, frac, _dp(out))
    return out


def profile_gh(z0, bin_dz, nbins, z1, zmax, lam, nmax, frac):
    arrs = [np.ascontiguousarray(a, dtype=np.float64) for a in (z1, zmax, lam, nmax)]
    out = np.zeros(nbins)
    lib().orc_profile_gh(z0, bin_dz, nbins, arrs[0].size, *[_dp(a) for a in arrs], frac, _dp(out))
    return out


def lateral_gaussian(L, sigma_cells):
    out = np.zeros((2 * L + 1) ** 2)
    lib().orc_lateral_gaussian(L, sigma_cells, _dp(out))
    return out


def lateral_nkg(L, dx, r_moliere, age, nsub, r_cut):
    out = np.zeros((2 * L + 1) ** 2)
    lib().orc_lateral_nkg(L, dx, r_moliere, age, nsub, r_cut, _dp(out))
    return out


def tables(w):
    """Profile and lateral tables of a ``workloads.Workload``, built by the
    oracle's own generators."""
    p, lt = w.profile, w.lateral
    if p["kind"] == "gaussian":
        q = profile_gaussian(w.z0, w.bin_dz, w.n_bins, p["z_peak"], p["l"], p["q_max"])
    elif p["kind"] == "greisen":
        q = profile_greisen(w.z0, w.bin_dz, w.n_bins, p["E0_eV"], p["Ec_eV"], p["X0_m"], p["frac"])
    elif p["kind"] == "gh":
        q = profile_gh(w.z0, w.bin_dz, w.n_bins, p["z1"], p["zmax"], p["lam"], p["nmax"], p["frac"])
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


def from_workload(w, max_steps=None):
    """An Oracle set up with the workload's grid, shower and detectors."""
    o = Oracle(w.nx, w.ny, w.nz, w.dx, w.dt, w.eps_r, w.boundary, w.npml)
    q, lw = tables(w)
    o.set_shower(q, w.z0, w.bin_dz, w.v, lw, w.lateral["L"])
    o.set_probes(w.probes_xyz, w.steps if max_steps is None else max_steps)
    return o


def set_threads(n: int = 0) -> int:
    """Threads of the oracle's parallel loops from now on (n >= 1); n <= 0
    leaves them unchanged.  Returns the count in force."""
    return int(lib().orc_set_threads(int(n)))
