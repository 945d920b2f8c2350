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
