"""Seeded synthetic inputs shared by the CUDA path, the oracle and the tests.

This module holds inputs only: grid sizes, time step, medium, the random draws
of the shower parameters and of the detector positions.  It holds none of the
method's arithmetic (no field update, no deposit, no profile formula); the
CUDA library and the oracle each turn these parameters into profile and
lateral tables with their own code.

The paper uses a parameterised shower instead of Monte Carlo output
(Sec. III.B), so every workload is synthetic:

* ``parity96``   96^3 cells, dx = 2 cm, Mur-1, 400 steps; Gaussian longitudinal
                 profile (l = 0.25 m, peak mid-grid, Q_max = -1 nC); Gaussian
                 lateral weights (1 cell, |di|,|dj| <= 4); 8 detectors at
                 R in [0.3, 0.9] m, theta in [30, 150] deg around the shower
                 maximum (seed 1001).
* ``greisen384`` 384x384x1536 cells, dx = 2 cm, 10-cell CPML, 4000 steps;
                 Greisen profile with E0 = 10^U[16,18] eV (seed 2002), 20 %
                 charge excess, NKG lateral spread (r_M = 10 cm); 64 detectors
                 at r in [1, 5] m along the shower.
* ``gh640``      640x640x2048 cells, dx = 3 cm, 12-cell CPML, 6000 steps; a sum
                 of 3-6 Gaisser-Hillas subshowers spread over 40 m (seed 3003);
                 256 detectors at r in [2, 10] m.

2D axisymmetric grids (the paper's own formulation, Table I):

* ``cyl_table1(n)`` n x n cells (nr = nz = n) over 40.96 m x 40.96 m, half the
                 2D Courant step, Mur-1, n steps (Table I's rates grow as
                 N_side, read as one step per cell of the side); the paper's
                 Gaussian shower model (Sec. III.B: longitudinal l = 2 m,
                 radial sigma_r = 5 cm) as the parameters of a 256-bin
                 charge table and of the ring weights, moving at c from 8 l
                 before its maximum; 64 detectors at R in [2, 0.4 n d] m,
                 theta in [40, 70] deg around the maximum (seed 4004).  The
                 2D solver takes tables; the library and the oracle build
                 them from these parameters with their own code.
* ``cyl_field(seed, comp, i, j, xp)`` counter-based initial field values
                 (uniform in [-1/2, 1/2), E in V/m, H_phi divided by the
                 impedance of ice), computable on any patch with NumPy or
                 torch with identical float32 results.

``scaled(...)`` shrinks a workload to a grid the oracle finishes in seconds
while keeping its physics (dx, dt, boundary, profile family, lateral family).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Optional

import numpy as np

C0 = 299792458.0          # m/s
EPS_R_ICE = 3.17          # relative permittivity of ice at radio frequencies
E_CRIT_ICE_EV = 78.6e6    # critical energy of electrons in ice, eV
X0_ICE_M = 36.08 / 0.918 / 100.0   # radiation length 36.08 g/cm^2 at 0.918 g/cm^3, in m
CHARGE_EXCESS = 0.2       # net charge / shower particles (Sec. I)
R_MOLIERE_M = 0.10        # lateral scale of the NKG spread

PEC, MUR1, CPML = 0, 1, 2


def courant_dt(dx: float, eps_r: float) -> float:
    """dt = 0.5 dx sqrt(eps_r) / (c sqrt 3): half the 3D Courant limit."""
    return 0.5 * dx * math.sqrt(eps_r) / (C0 * math.sqrt(3.0))


@dataclasses.dataclass
class Workload:
    name: str
    nx: int
    ny: int
    nz: int
    dx: float
    dt: float
    eps_r: float
    boundary: int
    npml: int
    steps: int
    # source: longitudinal profile parameters; tables are built by each side
    profile: dict
    lateral: dict
    z0: float
    bin_dz: float
    n_bins: int
    v: float
    probes_xyz: np.ndarray  # (n, 3) metres from node (0,0,0)

    @property
    def cells(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def cell_updates(self) -> int:
        return self.cells * self.steps

    def describe(self) -> dict:
        b = {PEC: "pec", MUR1: "mur1", CPML: f"cpml{self.npml}"}[self.boundary]
        return {"workload": self.name, "grid": [self.nx, self.ny, self.nz], "dx_m": self.dx,
                "dt_s": self.dt, "eps_r": self.eps_r, "boundary": b, "steps": self.steps,
                "profile": self.profile.get("kind"), "lateral": self.lateral.get("kind"),
                "probes": int(self.probes_xyz.shape[0])}


def _interior(nx, ny, nz, P):
    lo = P + 1
    return lo, nx - lo, lo, ny - lo, lo, nz - lo


def _snap_ok(x, y, z, dx, box):
    i, j, k = (math.floor(c / dx + 0.5) for c in (x, y, z))
    return box[0] <= i <= box[1] and box[2] <= j <= box[3] and box[4] <= k <= box[5]


def _probes_spherical(rng, n, centre, R_lo, R_hi, th_lo, th_hi, dx, box):
    """Detectors at (R, theta, phi) around the shower maximum (Sec. III.B)."""
    out = []
    while len(out) < n:
        R = rng.uniform(R_lo, R_hi)
        th = math.radians(rng.uniform(th_lo, th_hi))
        ph = rng.uniform(0.0, 2.0 * math.pi)
        x = centre[0] + R * math.sin(th) * math.cos(ph)
        y = centre[1] + R * math.sin(th) * math.sin(ph)
        z = centre[2] + R * math.cos(th)
        if _snap_ok(x, y, z, dx, box):
            out.append((x, y, z))
    return np.array(out, dtype=np.float64)


def _probes_cylindrical(rng, n, axis_xy, r_lo, r_hi, z_lo, z_hi, dx, box, max_tries=1000000):
    """Detectors at cylindrical radius r about the axis, uniform z and phi;
    draws whose node falls outside the non-PML interior are redrawn."""
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise ValueError("detector ring does not fit inside the grid interior")
        r = rng.uniform(r_lo, r_hi)
        ph = rng.uniform(0.0, 2.0 * math.pi)
        z = rng.uniform(z_lo, z_hi)
        x = axis_xy[0] + r * math.cos(ph)
        y = axis_xy[1] + r * math.sin(ph)
        if _snap_ok(x, y, z, dx, box):
            out.append((x, y, z))
    return np.array(out, dtype=np.float64)


def parity96(seed: int = 1001, n: int = 96, steps: int = 400, n_probes: int = 8) -> Workload:
    dx = 0.02
    dt = courant_dt(dx, EPS_R_ICE)
    rng = np.random.default_rng(seed)
    centre = ((n // 2) * dx, (n // 2) * dx, (n // 2) * dx)
    box = _interior(n, n, n, 0)
    scale = n / 96.0
    probes = _probes_spherical(rng, n_probes, centre, 0.3 * scale, 0.9 * scale, 30.0, 150.0, dx, box)
    return Workload(
        name=f"parity{n}", nx=n, ny=n, nz=n, dx=dx, dt=dt, eps_r=EPS_R_ICE, boundary=MUR1,
        npml=0, steps=steps,
        profile={"kind": "gaussian", "z_peak": centre[2], "l": 0.25 * scale, "q_max": -1e-9},
        lateral={"kind": "gaussian", "L": 4, "sigma_cells": 1.0},
        z0=0.0, bin_dz=dx / 4.0, n_bins=4 * n + 1, v=C0, probes_xyz=probes)


def greisen384(seed: int = 2002, nx: int = 384, ny: int = 384, nz: int = 1536, npml: int = 10,
               steps: int = 4000, n_probes: int = 64, r_lo: float = 1.0, r_hi: float = 5.0,
               E0: Optional[float] = None) -> Workload:
    dx = 0.02
    dt = courant_dt(dx, EPS_R_ICE)
    rng = np.random.default_rng(seed)
    if E0 is None:
        E0 = 10.0 ** rng.uniform(16.0, 18.0)
    z0 = (npml + 4) * dx
    z_end = (nz - npml) * dx
    n_bins = int(math.floor((z_end - z0) / (dx / 4.0))) + 1
    box = _interior(nx, ny, nz, npml)
    axis = ((nx // 2) * dx, (ny // 2) * dx)
    probes = _probes_cylindrical(rng, n_probes, axis, r_lo, r_hi, (npml + 1) * dx,
                                 (nz - npml - 1) * dx, dx, box)
    L = int(math.ceil(3.0 * R_MOLIERE_M / dx))
    return Workload(
        name=f"greisen{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, eps_r=EPS_R_ICE,
        boundary=CPML, npml=npml, steps=steps,
        profile={"kind": "greisen", "E0_eV": E0, "Ec_eV": E_CRIT_ICE_EV, "X0_m": X0_ICE_M,
                 "frac": CHARGE_EXCESS},
        lateral={"kind": "nkg", "L": L, "r_moliere": R_MOLIERE_M, "age": 1.0, "nsub": 4,
                 "r_cut": 3.0 * R_MOLIERE_M},
        z0=z0, bin_dz=dx / 4.0, n_bins=n_bins, v=C0, probes_xyz=probes)


def gh640(seed: int = 3003, nx: int = 640, ny: int = 640, nz: int = 2048, npml: int = 12,
          steps: int = 6000, n_probes: int = 256, r_lo: float = 2.0, r_hi: float = 10.0,
          spread_m: float = 40.0) -> Workload:
    dx = 0.03
    dt = courant_dt(dx, EPS_R_ICE)
    rng = np.random.default_rng(seed)
    nsub = int(rng.integers(3, 7))
    z0 = (npml + 4) * dx
    z1 = z0 + rng.uniform(0.0, spread_m, size=nsub)
    zmax = z1 + rng.uniform(3.0, 6.0, size=nsub)
    lam = rng.uniform(0.4, 0.8, size=nsub)
    nmax = 10.0 ** rng.uniform(8.0, 9.0, size=nsub)
    z_end = (nz - npml) * dx
    n_bins = int(math.floor((z_end - z0) / (dx / 4.0))) + 1
    box = _interior(nx, ny, nz, npml)
    axis = ((nx // 2) * dx, (ny // 2) * dx)
    probes = _probes_cylindrical(rng, n_probes, axis, r_lo, r_hi, (npml + 1) * dx,
                                 (nz - npml - 1) * dx, dx, box)
    L = int(math.ceil(3.0 * R_MOLIERE_M / dx))
    return Workload(
        name=f"gh{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, eps_r=EPS_R_ICE,
        boundary=CPML, npml=npml, steps=steps,
        profile={"kind": "gh", "z1": z1.tolist(), "zmax": zmax.tolist(), "lam": lam.tolist(),
                 "nmax": nmax.tolist(), "frac": CHARGE_EXCESS},
        lateral={"kind": "nkg", "L": L, "r_moliere": R_MOLIERE_M, "age": 1.0, "nsub": 4,
                 "r_cut": 3.0 * R_MOLIERE_M},
        z0=z0, bin_dz=dx / 4.0, n_bins=n_bins, v=C0, probes_xyz=probes)


def greisen_small(seed: int = 2002, nx: int = 64, ny: int = 56, nz: int = 200, npml: int = 10,
                  steps: int = 300, n_probes: int = 16) -> Workload:
    """The greisen384 physics on a grid the oracle finishes in seconds: same dx,
    dt, CPML depth, Greisen profile (the first nz cells of it) and NKG spread;
    detectors at r in [0.2, 0.45] m."""
    r_hi = min(0.45, (min(nx, ny) // 2 - npml - 2) * 0.02)
    w = greisen384(seed=seed, nx=nx, ny=ny, nz=nz, npml=npml, steps=steps, n_probes=n_probes,
                   r_lo=min(0.2, 0.5 * r_hi), r_hi=r_hi)
    w.name = f"greisen_small{nx}x{ny}x{nz}"
    return w


def gh_small(seed: int = 3003, nx: int = 60, ny: int = 52, nz: int = 160, npml: int = 12,
             steps: int = 250, n_probes: int = 16) -> Workload:
    """The gh640 physics (dx = 3 cm, 12-cell CPML, Gaisser-Hillas sum) on a
    small grid; subshowers spread over the short axis; r in [0.3, 0.45] m."""
    r_hi = min(0.45, (min(nx, ny) // 2 - npml - 2) * 0.03)
    w = gh640(seed=seed, nx=nx, ny=ny, nz=nz, npml=npml, steps=steps, n_probes=n_probes,
              r_lo=min(0.3, 0.5 * r_hi), r_hi=r_hi, spread_m=0.5 * nz * 0.03)
    # keep the subshowers short enough to develop inside the small grid
    p = w.profile
    rng = np.random.default_rng(seed + 1)
    n = len(p["z1"])
    p["zmax"] = (np.array(p["z1"]) + rng.uniform(0.3, 0.8, size=n)).tolist()
    p["lam"] = rng.uniform(0.1, 0.2, size=n).tolist()
    w.name = f"gh_small{nx}x{ny}x{nz}"
    return w


def surrogate_grid(nx: int = 128, ny: int = 128, nz: int = 512, npml: int = 10, steps: int = 2048,
                   n_bins: int = 128, m_steps: int = 8) -> Workload:
    """The grid of the surrogate's training runs: 128x128x512 cells, dx = 2 cm,
    10-cell CPML, 2048 steps; the profile is a 128-bin table from z0 =
    (npml + 4) dx whose bins are the distance the shower (v = c) covers in
    m_steps steps (8: 8.22 cm, 10.5 m in all); NKG lateral spread.  Shower and
    detectors are set per run (surrogate_runs)."""
    dx = 0.02
    dt = courant_dt(dx, EPS_R_ICE)
    bin_dz = m_steps * C0 * dt
    L = int(math.ceil(3.0 * R_MOLIERE_M / dx))
    return Workload(
        name=f"surrogate{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, eps_r=EPS_R_ICE,
        boundary=CPML, npml=npml, steps=steps,
        profile={"kind": "gh", "frac": CHARGE_EXCESS},
        lateral={"kind": "nkg", "L": L, "r_moliere": R_MOLIERE_M, "age": 1.0, "nsub": 4,
                 "r_cut": 3.0 * R_MOLIERE_M},
        z0=(npml + 4) * dx, bin_dz=bin_dz, n_bins=n_bins, v=C0, probes_xyz=np.zeros((0, 3)))


def surrogate_runs(seed: int, n_runs: int, n_probes: int = 64, grid: Optional[Workload] = None,
                   r_range=(0.3, 0.9), z_range=(0.5, 9.5), z1_range=(0.4, 2.0), len_range=(1.0, 3.5)) -> list:
    """Seeded draws of the surrogate's training runs: per run one Gaisser-Hillas
    shower (start z1 ~ z0 + U[z1_range] m, z_max - z1 ~ U[len_range] m,
    lambda ~ U[0.25, 0.6] m, N_max ~ 10^U[8, 9]) and n_probes detectors at
    r ~ U[r_range], z ~ U[z_range] (metres), phi ~ U[0, 2 pi) about the axis."""
    g = grid if grid is not None else surrogate_grid()
    rng = np.random.default_rng(seed)
    box = _interior(g.nx, g.ny, g.nz, g.npml)
    axis = ((g.nx // 2) * g.dx, (g.ny // 2) * g.dx)
    runs = []
    for _ in range(n_runs):
        z1 = g.z0 + rng.uniform(*z1_range)
        zmax = z1 + rng.uniform(*len_range)
        lam = rng.uniform(0.25, 0.6)
        nmax = 10.0 ** rng.uniform(8.0, 9.0)
        probes = _probes_cylindrical(rng, n_probes, axis, r_range[0], r_range[1], z_range[0], z_range[1], g.dx, box)
        runs.append({"z1": [z1], "zmax": [zmax], "lam": [lam], "nmax": [nmax], "probes_xyz": probes})
    return runs


def surrogate_lattice_grid(nx: int = 128, ny: int = 128, nz: int = 512, npml: int = 10, steps: int = 2048,
                           n_bins: int = 128, cells_per_bin: int = 4) -> Workload:
    """The grid of the lattice surrogate's FDTD runs: 128x128x512 cells, dx =
    2 cm, 10-cell CPML, 2048 steps, with the time step dt = dx / (2c), so that
    the shower (v = c) advances exactly half a cell per step (c' dt / dx =
    0.281, under the 3D Courant limit 0.577); 128 profile bins of 4 cells
    (8 steps) from z0 = (npml + 4) dx, covering 10.24 m; NKG lateral spread.
    Showers come from surrogate_runs, antennas from surrogate_lattice_antennas."""
    dx = 0.02
    dt = dx / (2.0 * C0)
    L = int(math.ceil(3.0 * R_MOLIERE_M / dx))
    return Workload(
        name=f"surrogate_lattice{nx}x{ny}x{nz}", nx=nx, ny=ny, nz=nz, dx=dx, dt=dt, eps_r=EPS_R_ICE,
        boundary=CPML, npml=npml, steps=steps,
        profile={"kind": "gh", "frac": CHARGE_EXCESS},
        lateral={"kind": "nkg", "L": L, "r_moliere": R_MOLIERE_M, "age": 1.0, "nsub": 4,
                 "r_cut": 3.0 * R_MOLIERE_M},
        z0=(npml + 4) * dx, bin_dz=cells_per_bin * dx, n_bins=n_bins, v=C0, probes_xyz=np.zeros((0, 3)))


def surrogate_lattice_antennas(grid: Workload, r_range=(0.3, 0.9), z_range=(0.5, 9.5), cells_per_bin: int = 4):
    """The antenna lattice of the surrogate: nodes in the half plane phi = 0
    (y on the axis, x = axis + i_r dx) with r = i_r dx in r_range, at the
    starts of the profile bins, z = z0 + cells_per_bin m dx in z_range.
    Returns (ir, m, xyz): radial class ir = i_r - i_r(min), bin index m, and
    the positions in metres (node coordinates from node (0, 0, 0))."""
    dx = grid.dx
    i_lo, i_hi = int(math.ceil(r_range[0] / dx - 1e-9)), int(math.floor(r_range[1] / dx + 1e-9))
    kz0 = int(round(grid.z0 / dx))
    m_lo = int(math.ceil((z_range[0] / dx - kz0) / cells_per_bin - 1e-9))
    m_hi = int(math.floor((z_range[1] / dx - kz0) / cells_per_bin + 1e-9))
    ic, jc = grid.nx // 2, grid.ny // 2
    ir, m = np.meshgrid(np.arange(i_hi - i_lo + 1), np.arange(m_lo, m_hi + 1), indexing="ij")
    ir, m = ir.ravel(), m.ravel()
    xyz = np.stack([(ic + i_lo + ir) * dx, np.full(ir.size, jc * dx), (kz0 + cells_per_bin * m) * dx], axis=1)
    return ir.astype(np.int32), m.astype(np.int32), xyz


@dataclasses.dataclass
class CylWorkload:
    name: str
    nr: int
    nz: int
    d: float
    dt: float
    eps_r: float
    boundary: int
    steps: int
    shower: dict           # Gaussian model parameters: z_peak, l, q_max (C), n_bins,
                           # sigma_r (m), n_rings; tables are built by each side
    z0: float              # position of bin 0 (m)
    bin_dz: float
    v: float
    probes_rz: np.ndarray  # [n, 2] (r, z) in metres

    @property
    def cells(self) -> int:
        return self.nr * self.nz

    def describe(self) -> dict:
        return {"workload": self.name, "grid_rz": [self.nr, self.nz], "d_m": self.d, "dt_s": self.dt,
                "eps_r": self.eps_r, "boundary": {PEC: "pec", MUR1: "mur1"}[self.boundary],
                "steps": self.steps, "rings": int(self.shower["n_rings"]), "probes": int(len(self.probes_rz))}


def courant_dt_2d(d: float, eps_r: float) -> float:
    """dt = 0.5 d sqrt(eps_r) / (c sqrt 2): half the 2D Courant limit."""
    return 0.5 * d * math.sqrt(eps_r) / (C0 * math.sqrt(2.0))


def cyl_table1(n: int = 8192, seed: int = 4004, extent_m: float = 40.96, steps: Optional[int] = None,
               n_probes: int = 64, l_m: float = 2.0, sigma_r_m: float = 0.05, q_max: float = -1e-9,
               boundary: int = MUR1) -> CylWorkload:
    d = extent_m / n
    dt = courant_dt_2d(d, EPS_R_ICE)
    rng = np.random.default_rng(seed)
    z_max = extent_m * (0.45 + 0.1 * rng.random())
    n_bins = 256
    z0 = z_max - 4.0 * l_m
    bin_dz = 8.0 * l_m / (n_bins - 1)
    # rings out to 3 sigma_r (ring i covers [(i - 1/2) d, (i + 1/2) d])
    n_rings = max(1, min(n, int(math.ceil(3.0 * sigma_r_m / d)) + 1))
    shower = {"kind": "gaussian", "z_peak": z_max, "l": l_m, "q_max": q_max, "n_bins": n_bins,
              "sigma_r": sigma_r_m, "n_rings": n_rings}
    R = rng.uniform(min(2.0, 0.1 * extent_m), 0.4 * extent_m, n_probes)
    th = np.radians(rng.uniform(40.0, 70.0, n_probes))
    rz = np.stack([R * np.sin(th), z_max + R * np.cos(th)], axis=1)
    rz[:, 0] = np.clip(rz[:, 0], 0.0, (n - 1) * d)
    rz[:, 1] = np.clip(rz[:, 1], d, (n - 1) * d)
    return CylWorkload(f"cyl{n}x{n}", n, n, d, dt, EPS_R_ICE, boundary, n if steps is None else steps,
                       shower, z0, bin_dz, C0, rz)


Z_ICE = 376.730313668 / math.sqrt(EPS_R_ICE)


def cyl_field(seed: int, comp: int, i, j, xp=np):
    """Initial value of component comp (0 E_r, 1 E_z, 2 H_phi) at integer
    indices i, j (broadcast arrays of NumPy or torch int64): a 32-bit
    multiply-xorshift hash of (seed, comp, i, j) mapped to [-1/2, 1/2), H_phi
    divided by Z_ICE.  Identical float32 values from NumPy and torch."""
    M = 0xFFFFFFFF
    x = (i * 0x9E3779B1 + (j + 0x632BE5AB) * 0x85EBCA77 + (seed * 4 + comp) * 0xC2B2AE3D) & M
    for _ in range(3):
        x = x ^ (x >> 15)
        x = (x * 0x2C1B3C6D) & M
        x = x ^ (x >> 12)
        x = (x * 0x297A2D39) & M
    x = x ^ (x >> 15)
    f = (x >> 8)
    if xp is np:
        v = f.astype(np.float32) * np.float32(2.0 ** -24) - np.float32(0.5)
        return v / np.float32(Z_ICE) if comp == 2 else v
    v = f.to(xp.float32) * (2.0 ** -24) - 0.5
    return v / Z_ICE if comp == 2 else v


WORKLOADS = {"parity96": parity96, "greisen384": greisen384, "gh640": gh640,
             "greisen_small": greisen_small, "gh_small": gh_small, "surrogate_grid": surrogate_grid,
             "surrogate_lattice_grid": surrogate_lattice_grid}
