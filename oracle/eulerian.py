"""Riemann-based Eulerian weakly-compressible SPH of the oracle (test infrastructure).

Sec. 3.1.  Particles do not move; each carries a fixed volume w_i = V_i (here the
caller's ``vol``), a density rho_i = rho0 + drho_i and a velocity v_i.  With the
weakly-compressible equation of state p = c0^2 (rho - rho0) (Sec. 3.1.1) the
energy equation is inactive and Eq. 18 reduces to (dividing by the constant w_i)

    d rho_i / dt     = -2 sum_j V_j rho*  (v* . g_ij)
    d (rho v)_i / dt = -2 sum_j V_j [rho* v* (v* . g_ij) + p* g_ij]  (+ viscosity)

with the corrected gradient g_ij = (B_i + B_j)/2 grad W_ij of Eq. 27 and the
star states of the linearised Riemann solver with the dissipation limiter,
Eqs. 25-26 (eta = 15):

    beta = min(eta max((u_l - u_r)/c, 0), 1)
    u*   = (u_l + u_r)/2 + beta^2 (p_l - p_r) / (2 rho_bar c)
    p*   = (p_l + p_r)/2 + beta rho_bar c (u_l - u_r) / 2

Readings (the paper leaves these open):
* left = i, right = j, normal n = -e_ij (pointing from i to j), u_l = v_i.n,
  u_r = v_j.n, rho_bar = (rho_i + rho_j)/2, c_bar = c0 (constant sound speed);
* the star velocity keeps the mean tangential part, v* = v_bar + (u* - u_bar) n,
  following the HLLC tangential rule of Eq. 21, and rho* = rho_bar;
* Eq. 25 is used as printed: beta^2 on the pressure jump in u*, beta in p*;
* viscosity (the paper's viscous cases give no discretisation) is the
  Morris-type term 2 mu sum_j V_j (v_i - v_j)(r_ij . grad W_ij)/(r^2 + 0.01 h^2)
  with the uncorrected (truncated) gradient, added to d(rho v)/dt;
* time integration (not stated): a momentum pass with (rho^n, v^n) gives
  (rho v)^{n+1} and v' = (rho v)^{n+1}/rho^n; a continuity pass with
  (rho^n, v') gives rho^{n+1}; then v^{n+1} = (rho v)^{n+1}/rho^{n+1}.  The
  single-pass forward-Euler variant evaluates both rates at (rho^n, v^n).
"""
from dataclasses import dataclass

import numpy as np

from .kgc import kernel_gradients, sym_to_full
from .kernels import WENDLAND


@dataclass
class EulerianParams:
    dom: object          # neighbors.Domain (kappa = 1.6 or 2)
    dt: float
    rho0: float = 1.0
    c0: float = 10.0
    mu: float = 0.0
    eta: float = 15.0


def pressure(drho, c0):
    """Weakly-compressible EOS, Sec. 3.1.1: p = c0^2 (rho - rho0)."""
    return c0 * c0 * drho


def acoustic_star_state(ul, ur, pl, pr, rho_bar, c_bar, eta):
    """Linearised Riemann solver with the dissipation limiter, Eqs. 25-26."""
    beta = np.minimum(eta * np.maximum((ul - ur) / c_bar, 0.0), 1.0)
    ustar = 0.5 * (ul + ur) + 0.5 * beta * beta * (pl - pr) / (rho_bar * c_bar)
    pstar = 0.5 * (pl + pr) + 0.5 * beta * rho_bar * c_bar * (ul - ur)
    return ustar, pstar


def eulerian_rates(pos, vol, drho, v, Bs, row_ptr, col, prm, want_mass=True, want_mom=True):
    """Right-hand sides of Eq. 18 (mass and momentum rows) at the given state.

    Returns (d rho/dt of shape (n,), d(rho v)/dt of shape (dim, n))."""
    dom = prm.dom
    dim = dom.dim
    n = pos.shape[1]
    i, j, rij, r, grad = kernel_gradients(pos, row_ptr, col, dom, WENDLAND)
    B = sym_to_full(Bs, dim)
    Bbar = 0.5 * (B[i] + B[j])                      # (m, d, d)
    g = np.einsum("mab,bm->am", Bbar, grad)          # Eq. 27
    nrm = -rij / r                                   # from i towards j
    vi = v[:, i]
    vj = v[:, j]
    ul = np.sum(vi * nrm, axis=0)
    ur = np.sum(vj * nrm, axis=0)
    rho_i = prm.rho0 + drho[i]
    rho_j = prm.rho0 + drho[j]
    p_i = pressure(drho[i], prm.c0)
    p_j = pressure(drho[j], prm.c0)
    rho_bar = 0.5 * (rho_i + rho_j)
    ustar, pstar = acoustic_star_state(ul, ur, p_i, p_j, rho_bar, prm.c0, prm.eta)
    ubar = 0.5 * (ul + ur)
    vstar = 0.5 * (vi + vj) + (ustar - ubar) * nrm
    rhostar = rho_bar
    vg = np.sum(vstar * g, axis=0)
    vj_w = vol[j]
    drho_dt = np.zeros(n)
    dmom_dt = np.zeros((dim, n))
    if want_mass:
        drho_dt = -2.0 * np.bincount(i, weights=vj_w * rhostar * vg, minlength=n)
    if want_mom:
        visc_w = None
        if prm.mu != 0.0:
            rdotg = np.sum(rij * grad, axis=0)
            visc_w = 2.0 * prm.mu * vj_w * rdotg / (r * r + 0.01 * dom.h * dom.h)
        for a in range(dim):
            flux = rhostar * vstar[a] * vg + pstar * g[a]
            dmom_dt[a] = -2.0 * np.bincount(i, weights=vj_w * flux, minlength=n)
            if visc_w is not None:
                dmom_dt[a] += np.bincount(i, weights=visc_w * (vi[a] - vj[a]), minlength=n)
    return drho_dt, dmom_dt


def step_two_pass(pos, vol, drho, v, Bs, row_ptr, col, prm):
    """One time step: momentum pass, then continuity pass with the new velocity."""
    rho_n = prm.rho0 + drho
    _, dmom = eulerian_rates(pos, vol, drho, v, Bs, row_ptr, col, prm, want_mass=False)
    mom1 = rho_n * v + prm.dt * dmom
    v_half = mom1 / rho_n
    drho_dt, _ = eulerian_rates(pos, vol, drho, v_half, Bs, row_ptr, col, prm, want_mom=False)
    drho1 = drho + prm.dt * drho_dt
    v1 = mom1 / (prm.rho0 + drho1)
    return drho1, v1


def step_fused(pos, vol, drho, v, Bs, row_ptr, col, prm):
    """One forward-Euler step with both rates at (rho^n, v^n)."""
    rho_n = prm.rho0 + drho
    drho_dt, dmom = eulerian_rates(pos, vol, drho, v, Bs, row_ptr, col, prm)
    mom1 = rho_n * v + prm.dt * dmom
    drho1 = drho + prm.dt * drho_dt
    return drho1, mom1 / (prm.rho0 + drho1)


def run(pos, vol, drho, v, Bs, row_ptr, col, prm, nsteps, fused=False):
    step = step_fused if fused else step_two_pass
    for _ in range(nsteps):
        drho, v = step(pos, vol, drho, v, Bs, row_ptr, col, prm)
    return drho, v


def time_step(h, c0, U, mu, rho0):
    """Fixed step: acoustic limit 0.25 h/(c0 + U) and viscous limit 0.125 h^2 rho0/mu."""
    dt = 0.25 * h / (c0 + U)
    if mu > 0.0:
        dt = min(dt, 0.125 * h * h * rho0 / mu)
    return dt
