"""FP64 CPU oracle of the paper's 2D axisymmetric FDTD (E_r, E_z, H_phi) --
TEST INFRASTRUCTURE.

Only tests/, __graft_entry__.smoke() and bench.py's reference legs may use
this module.  It shares no code with the CUDA library (csrc/cyl.cu); the two
meet only through seeded inputs.

The paper assumes cylindrical symmetry about the shower axis (Sec. III.A): the
phi derivatives vanish, H_r, H_z and E_phi vanish, and Maxwell's equations
reduce to
    eps dE_r/dt = -dH_phi/dz - J_r,
    eps dE_z/dt = (1/r) d(r H_phi)/dr - J_z,
    mu dH_phi/dt = -(dE_r/dz - dE_z/dr)        (Eqs. fdtd_Er, fdtd_Ez, fdtd_Hphi, sigma = 0).
Discretisation (central differences, second order in space and time; the
paper updates E then H, here H^{n+1/2} then E^{n+1}, the same leapfrog):
  nodes r = i d (i = 0..nr), z = j d (j = 0..nz);
  E_r at (i+1/2, j), E_z at (i, j+1/2), H_phi at (i+1/2, j+1/2);
  H_phi -= dt/(mu d) [E_r(i+1/2, j+1) - E_r(i+1/2, j) - E_z(i+1, j+1/2) + E_z(i, j+1/2)];
  E_r  -= dt/(eps d) [H_phi(i+1/2, j+1/2) - H_phi(i+1/2, j-1/2)] + dt J_r / eps      (0 < j < nz);
  E_z  += dt/(eps d r_i) [r_{i+1/2} H_phi(i+1/2, j+1/2) - r_{i-1/2} H_phi(i-1/2, j+1/2)] - dt J_z / eps
          (0 < i < nr); on the axis (Ampere's law over the disc of radius d/2)
  E_z(0, j+1/2) += 4 dt/(eps d) H_phi(1/2, j+1/2) - dt J_z / eps.
The outer wall (r = nr d) and the end caps (z = 0, nz d) are PEC, or carry
first-order Mur on their tangential E (E_z at the wall, E_r at the caps).

Source (reading, as in the 3D path): the shower's charge q(z_s) at
z_s = z0 + v t, spread over rings with weights w_i (sum 1, ring i covering
r in [(i-1/2) d, (i+1/2) d], the axis disc [0, d/2]), moves along the axis
as a cloud-in-cell line; the current density through the face (i, j+1/2) is
the charge that crossed it,
    J_z = -(d/dt) qbar w_i [C_j(z^{n+1}) - C_j(z^n)] / (A_i d),
with qbar = q(z_s^{n+1/2}) (linear in a bin table), C_j the cumulative CIC
weight of the nodes <= j, and A_i the ring's cross-section (pi d^2/4 on the
axis, 2 pi r_i d elsewhere); J_r = 0.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)
PEC, MUR1 = 0, 1


def ring_area(nr, d, i0=0):
    """Cross-section of the rings of rows i0 .. i0+nr (axis disc pi d^2 / 4)."""
    A = 2.0 * math.pi * (i0 + np.arange(nr + 1)) * d * d
    if i0 == 0:
        A[0] = math.pi * d * d / 4.0
    return A


class CylOracle:
    def __init__(self, nr, nz, d, dt, eps_r, boundary=MUR1, i0=0):
        """i0 > 0: the grid is the patch of rows i0 .. i0+nr of a larger grid
        (radii (i0 + i) d); its row 0 is then not the axis and its E_z is held
        fixed, so only cells whose dependency cone stays inside the patch are
        those of the larger grid."""
        self.nr, self.nz, self.d, self.dt = nr, nz, d, dt
        self.i0 = int(i0)
        self.eps = eps_r * EPS0
        self.boundary = boundary
        self.Er = np.zeros((nr, nz + 1))        # (i+1/2, j)
        self.Ez = np.zeros((nr + 1, nz))        # (i, j+1/2)
        self.Hp = np.zeros((nr, nz))            # (i+1/2, j+1/2)
        self.steps = 0
        self.src = None
        self.probes = np.zeros((0, 2), dtype=np.int64)
        self.trace = []
        S = C0 / math.sqrt(eps_r) * dt / d
        self.mur = (S - 1.0) / (S + 1.0)

    # ---- source -------------------------------------------------------------
    def set_shower(self, q, z0, bin_dz, v, w):
        """q: charge per bin (C) at z0 + b bin_dz (linear in between);
        w: ring weights w_i, i < len(w) (sum 1)."""
        self.src = (np.asarray(q, dtype=np.float64), float(z0), float(bin_dz), float(v),
                    np.asarray(w, dtype=np.float64))

    def _q(self, z):
        q, z0, bdz, _, _ = self.src
        x = (z - z0) / bdz
        if x < 0 or x > len(q) - 1:
            return 0.0
        b = min(int(math.floor(x)), len(q) - 2)
        f = x - b
        return (1 - f) * q[b] + f * q[b + 1]

    def _cum(self, zs):
        """C_j for all j: cumulative CIC weight of the nodes <= j of a unit
        charge at zs (nodes z = j d, j = 0..nz)."""
        x = zs / self.d
        j = math.floor(x)
        f = x - j
        C = np.zeros(self.nz + 1)
        # node j gets 1-f, node j+1 gets f
        C[np.arange(self.nz + 1) >= j] += 1 - f
        C[np.arange(self.nz + 1) >= j + 1] += f
        return C

    def current(self):
        """J_z at faces (i, j+1/2), [nr+1, nz], for the step n -> n+1."""
        J = np.zeros((self.nr + 1, self.nz))
        if self.src is None:
            return J
        q, z0, bdz, v, w = self.src
        n = self.steps
        za, zb = z0 + v * n * self.dt, z0 + v * (n + 1) * self.dt
        qbar = self._q(z0 + v * (n + 0.5) * self.dt)
        if qbar == 0.0:
            return J
        dC = (self._cum(zb) - self._cum(za))[:self.nz]          # crossing of face j+1/2
        A = ring_area(self.nr, self.d, self.i0)
        for i in range(self.nr + 1):
            if self.i0 + i < len(w):
                J[i] = -(self.d / self.dt) * qbar * w[self.i0 + i] * dC / (A[i] * self.d)
        return J

    # ---- detectors ------------------------------------------------------------
    def set_probes(self, rz):
        """Detectors at (r, z) in metres, snapped to the nearest node; each
        reading is (E_z, E_r) at the node: E_z averaged over j+-1/2, E_r over
        i+-1/2 (E_r = 0 on the axis)."""
        rz = np.asarray(rz, dtype=np.float64).reshape(-1, 2)
        self.probes = np.floor(rz / self.d + 0.5).astype(np.int64)
        if np.any(self.probes[:, 0] < 0) or np.any(self.probes[:, 0] >= self.nr) or \
                np.any(self.probes[:, 1] < 1) or np.any(self.probes[:, 1] >= self.nz):
            raise ValueError("detector outside the grid interior")
        self.trace = []

    def _read(self):
        out = np.zeros((len(self.probes), 2))
        for p, (i, j) in enumerate(self.probes):
            ez = 0.5 * (self.Ez[i, j - 1] + self.Ez[i, j])
            er = 0.0 if i == 0 else 0.5 * (self.Er[i - 1, j] + self.Er[i, j])
            out[p] = (ez, er)
        return out

    # ---- step -----------------------------------------------------------------
    def step(self, n=1):
        d, dt, eps = self.d, self.dt, self.eps
        nr, nz = self.nr, self.nz
        r_half = (self.i0 + np.arange(nr) + 0.5) * d          # r_{i+1/2}
        r_node = (self.i0 + np.arange(nr + 1)) * d
        for _ in range(n):
            J = self.current()
            Er0, Ez0 = self.Er.copy(), self.Ez.copy()
            # H^{n+1/2}
            self.Hp -= dt / (MU0 * d) * ((self.Er[:, 1:] - self.Er[:, :-1]) - (self.Ez[1:, :] - self.Ez[:-1, :]))
            # E^{n+1}
            self.Er[:, 1:nz] -= dt / (eps * d) * (self.Hp[:, 1:] - self.Hp[:, :-1])
            rH = r_half[:, None] * self.Hp
            self.Ez[1:nr, :] += dt / (eps * d * r_node[1:nr, None]) * (rH[1:, :] - rH[:-1, :])
            if self.i0 == 0:
                self.Ez[0, :] += 4.0 * dt / (eps * d) * self.Hp[0, :]
                self.Ez -= dt / eps * J
            else:
                self.Ez[1:] -= dt / eps * J[1:]
            if self.boundary == MUR1:
                m = self.mur
                # wall r = nr d: E_z(nr, j+1/2) from E_z(nr-1, .)
                self.Ez[nr, :] = Ez0[nr - 1, :] + m * (self.Ez[nr - 1, :] - Ez0[nr, :])
                # caps z = 0 and nz d: E_r(i+1/2, 0) and (i+1/2, nz)
                self.Er[:, 0] = Er0[:, 1] + m * (self.Er[:, 1] - Er0[:, 0])
                self.Er[:, nz] = Er0[:, nz - 1] + m * (self.Er[:, nz - 1] - Er0[:, nz])
            else:
                self.Ez[nr, :] = 0.0
                self.Er[:, 0] = 0.0
                self.Er[:, nz] = 0.0
            self.steps += 1
            if len(self.probes):
                self.trace.append(self._read())

    def traces(self):
        """[n_probes][steps][2] (E_z, E_r)."""
        if not self.trace:
            return np.zeros((len(self.probes), 0, 2))
        return np.stack(self.trace, axis=1)

    # ---- diagnostics ----------------------------------------------------------
    def divergence(self):
        """eps * discrete div E at the nodes (i, j), 0 < j < nz, 0 <= i < nr
        (ring-volume form: flux through the node's ring faces / ring volume)."""
        d, nr, nz = self.d, self.nr, self.nz
        A = ring_area(nr, d)                                # axial faces of node i's ring
        side = 2.0 * math.pi * (np.arange(nr) + 0.5) * d * d   # outer radial face of ring i
        V = A * d                                           # ring volumes
        div = np.zeros((nr, nz + 1))
        for i in range(nr):
            flux = A[i] * (self.Ez[i, 1:nz] - self.Ez[i, 0:nz - 1])
            flux = np.concatenate([[0.0], flux, [0.0]])
            flux += side[i] * self.Er[i, :]
            if i > 0:
                flux -= side[i - 1] * self.Er[i - 1, :]
            div[i] = flux / V[i]
        return self.eps * div

    def energy(self):
        """Electric energy 1/2 eps sum E^2 dV over the ring volumes of the
        components (and magnetic energy of H^{n-1/2} the same way)."""
        d, nr = self.d, self.nr
        Vr = 2.0 * math.pi * ((np.arange(nr) + 0.5) * d) * d * d
        Vz = ring_area(nr, d) * d
        Vh = Vr
        We = 0.5 * self.eps * ((Vr[:, None] * self.Er ** 2).sum() + (Vz[:, None] * self.Ez ** 2).sum())
        Wh = 0.5 * MU0 * (Vh[:, None] * self.Hp ** 2).sum()
        return We, Wh


def courant_dt(d, eps_r):
    """Half of the 2D Courant limit d sqrt(eps_r) / (c sqrt 2)."""
    return 0.5 * d * math.sqrt(eps_r) / (C0 * math.sqrt(2.0))


def ring_weights_gaussian(n_rings, d, sigma_r):
    """Share of a radial Gaussian charge density exp(-r^2 / (2 sigma_r^2))
    (the paper's lateral model, Sec. III.B) in each ring i: r in
    [(i-1/2) d, (i+1/2) d], the axis disc [0, d/2] for i = 0; renormalised to
    sum 1 over the n_rings rings.  The charge inside radius r is
    1 - exp(-r^2 / (2 sigma_r^2)) of the total (the integral of the density
    over the disc)."""
    edges = np.concatenate([[0.0], (np.arange(n_rings) + 0.5) * d])
    inside = 1.0 - np.exp(-0.5 * (edges / sigma_r) ** 2)
    w = np.diff(inside)
    return w / w.sum()


def tables(w):
    """Charge table (Eq. showerModel, sampled by the 3D oracle's generator) and
    ring weights of a ``workloads.CylWorkload``, built on the oracle side."""
    import oracle
    s = w.shower
    if s["kind"] != "gaussian":
        raise ValueError(s["kind"])
    q = oracle.profile_gaussian(w.z0, w.bin_dz, s["n_bins"], s["z_peak"], s["l"], s["q_max"])
    return q, ring_weights_gaussian(s["n_rings"], w.d, s["sigma_r"])
