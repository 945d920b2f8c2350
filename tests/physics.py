"""Closed forms and invariants the FDTD results are checked against.

Independent of both the oracle and the CUDA library: nothing here steps a
grid.  Used by the tests only.
"""
from __future__ import annotations

import math

import numpy as np

C0 = 299792458.0
MU0 = 1.25663706212e-6
EPS0 = 1.0 / (MU0 * C0 * C0)


def live_masks(nx, ny, nz, pec_tangential_zero=True):
    """Boolean masks (nz+1, ny+1, nx+1) of the entries each Yee component
    updates: Ex(i+1/2,j,k), Ey(i,j+1/2,k), Ez(i,j,k+1/2), Hx(i,j+1/2,k+1/2),
    Hy(i+1/2,j,k+1/2), Hz(i+1/2,j+1/2,k).  With ``pec_tangential_zero`` the
    E entries lying on the outer faces (tangential there) are excluded."""
    sh = (nz + 1, ny + 1, nx + 1)
    m = [np.zeros(sh, bool) for _ in range(6)]
    e0 = 1 if pec_tangential_zero else 0
    m[0][e0:nz + 1 - e0, e0:ny + 1 - e0, 0:nx] = True
    m[1][e0:nz + 1 - e0, 0:ny, e0:nx + 1 - e0] = True
    m[2][0:nz, e0:ny + 1 - e0, e0:nx + 1 - e0] = True
    m[3][0:nz, 0:ny, 0:nx + 1] = True
    m[4][0:nz, 0:ny + 1, 0:nx] = True
    m[5][0:nz + 1, 0:ny, 0:nx] = True
    return m


def discrete_omega(kvec, dx, dt, cp):
    """Yee dispersion relation: sin^2(w dt/2)/(c' dt)^2 = sum_d sin^2(k_d dx/2)/dx^2."""
    s = sum(math.sin(k * dx / 2.0) ** 2 for k in kvec) / dx ** 2
    return 2.0 / dt * math.asin(cp * dt * math.sqrt(s))


def cic_hat(u):
    """Linear charge-assignment weight of a node at distance u (in cells)."""
    return np.maximum(0.0, 1.0 - np.abs(u))


def gauss_filter_trace(trace, dt, sigma_t, t_samples, t0=0.0):
    """(g * x)(t) for a trace x_n at times t0 + n dt, g a unit-area Gaussian."""
    tn = t0 + dt * np.arange(trace.shape[-1])
    G = np.exp(-0.5 * ((t_samples[:, None] - tn[None, :]) / sigma_t) ** 2) / (math.sqrt(2 * math.pi) * sigma_t)
    return (G * dt) @ trace


def _phi(u):
    return np.exp(-0.5 * u * u) / math.sqrt(2.0 * math.pi)


def _Phi(u):
    from scipy.special import ndtr
    return ndtr(u)


def moving_charge_field(obs, z_src, q_src, t_src, t, eps, sigma_t):
    """Gaussian-filtered E field of a charge moving along the z axis, as the
    superposition of retarded Hertzian dipoles (the Green's-function solution
    of the inhomogeneous Maxwell equations, Sec. II, written in the time domain
    for a current I(z) dz = q(z) v).

    The path element at z' (length dz, charge q(z')) carries the dipole moment
    p(t) = q(z') dz H(t - t'(z')); filtered by a Gaussian of width sigma_t:
    p = Phi(u), pdot = phi(u)/sigma_t, pddot = -u phi(u)/sigma_t^2,
    u = (t - t' - R/c')/sigma_t.  Field of p z^ at distance R along r^:
    E = [ (3 (r^.z^) r^ - z^)(p/R^3 + pdot/(c'R^2)) + ((r^.z^) r^ - z^) pddot/(c'^2 R) ] / (4 pi eps).

    obs: (3,) observer position (axis at x = y = 0); z_src, q_src, t_src: the
    quadrature nodes (position, charge per node = q(z') dz, passage time);
    t: (nt,) observer times.  Returns (nt, 3)."""
    cp = 1.0 / math.sqrt(MU0 * eps)
    dxv = obs[0]
    dyv = obs[1]
    dzv = obs[2] - z_src                     # (nz,)
    R = np.sqrt(dxv * dxv + dyv * dyv + dzv * dzv)
    rx, ry, rz = dxv / R, dyv / R, dzv / R   # (nz,)
    u = (t[None, :] - t_src[:, None] - (R / cp)[:, None]) / sigma_t   # (nz, nt)
    p = _Phi(u)
    pd = _phi(u) / sigma_t
    pdd = -u * _phi(u) / sigma_t ** 2
    Rc = R[:, None]
    near = p / Rc ** 3 + pd / (cp * Rc ** 2)
    far = pdd / (cp * cp * Rc)
    cz = rz[:, None]
    out = np.zeros((t.size, 3))
    for comp, rc, zc in ((0, rx, 0.0), (1, ry, 0.0), (2, rz, 1.0)):
        rcc = rc[:, None]
        term = (3.0 * cz * rcc - zc) * near + (cz * rcc - zc) * far
        out[:, comp] = (q_src[:, None] * term).sum(axis=0)
    return out / (4.0 * math.pi * eps)


def nkg_norm(s):
    """Normalisation of the NKG lateral density: 2 pi int_0^inf x rho(x) dx = 1
    for rho(x) = C x^(s-2) (1+x)^(s-4.5), x = r/r_M:
    C = Gamma(4.5-s) / (2 pi Gamma(s) Gamma(4.5-2s))."""
    return math.gamma(4.5 - s) / (2.0 * math.pi * math.gamma(s) * math.gamma(4.5 - 2.0 * s))


# ---- frequency domain (Sec. II and V; E_w = int E(t) exp(+i w t) dt) ----------

def line_current_field_w(freqs, r_obs, z_obs, z_src, q_src, t_src, eps):
    """Exact E_omega = (E_z, E_r) at (r_obs, z_obs) of a current along the
    z axis (the solution of eq. GreenMethod for it), as the superposition of
    Hertzian elements.  A charge q(z') moving along the axis passes z' at t';
    its current is I_w dz' = q(z') dz' exp(i w t') per element (q_src holds
    q(z') dz').  An element at distance D and polar angle th (from +z):
        E_D  = eta (I dz) cos(th) / (2 pi D^2) (1 + i/(kD)) exp(ikD),
        E_th = -i eta k (I dz) sin(th) / (4 pi D) (1 + i/(kD) - 1/(kD)^2) exp(ikD),
    eta = sqrt(mu0/eps), k = w sqrt(mu0 eps).  Its charges (continuity) are
    part of this field, so the charge the shower leaves at rest is included.
    Returns two complex arrays [n_f]."""
    f = np.asarray(freqs, dtype=np.float64).ravel()
    w = 2.0 * math.pi * f
    k = w * math.sqrt(MU0 * eps)
    eta = math.sqrt(MU0 / eps)
    dz = z_obs - np.asarray(z_src, dtype=np.float64)
    D = np.sqrt(r_obs * r_obs + dz * dz)
    c, s = dz / D, r_obs / D
    kD = k[:, None] * D[None, :]
    ph = np.exp(1j * (kD + w[:, None] * np.asarray(t_src)[None, :])) * np.asarray(q_src)[None, :]
    ED = eta * c / (2 * math.pi * D * D) * (1 + 1j / kD) * ph
    Et = -1j * eta * k[:, None] * s / (4 * math.pi * D) * (1 + 1j / kD - 1 / (kD * kD)) * ph
    Ez = (ED * c - Et * s).sum(axis=1)
    Er = (ED * s + Et * c).sum(axis=1)
    return Ez, Er


def far_field_1d(freqs, theta, R, n_idx, z_rel, q_dz, t_ref=0.0, v=C0):
    """Eq. 1d_appro in its integral form: the theta-hat field of the
    Fraunhofer approximation (eq. fraun_appr) for a charge q(z') moving at v
    along the axis, the frame centred on the axis point that the charge
    passes at t_ref, z_rel = z' measured from it, q_dz = q(z') dz':
        E_theta = -i w mu0/(4 pi) sin(theta) exp(ikR)/R exp(i w t_ref)
                  * sum q(z') dz' exp(i p z'),   p = w (1/v - n cos(theta)/c).
    (The paper writes it with e N_e(z') for q(z') and the unit vector n_perp = -theta-hat.)"""
    f = np.asarray(freqs, dtype=np.float64).ravel()
    w = 2.0 * math.pi * f
    k = w * n_idx / C0
    p = w * (1.0 / v - n_idx * math.cos(theta) / C0)
    I = (np.asarray(q_dz)[None, :] * np.exp(1j * p[:, None] * np.asarray(z_rel)[None, :])).sum(axis=1)
    return -1j * w * MU0 / (4 * math.pi) * math.sin(theta) * np.exp(1j * (k * R + w * t_ref)) / R * I


def far_field_1d_gauss(freqs, theta, R, n_idx, q_max, l, t_ref=0.0, v=C0):
    """Eq. 1d_appro's closed form for the Gaussian profile q(z') = q_max
    exp(-z'^2 / (2 l^2)) of eq. showerModel: the integral is
    sqrt(2 pi) q_max l exp(-l^2 p^2 / 2)."""
    f = np.asarray(freqs, dtype=np.float64).ravel()
    w = 2.0 * math.pi * f
    k = w * n_idx / C0
    p = w * (1.0 / v - n_idx * math.cos(theta) / C0)
    I = math.sqrt(2 * math.pi) * q_max * l * np.exp(-0.5 * (l * p) ** 2)
    return -1j * w * MU0 / (4 * math.pi) * math.sin(theta) * np.exp(1j * (k * R + w * t_ref)) / R * I
