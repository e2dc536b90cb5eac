"""Riemann-based Eulerian SPH for compressible flow, oracle version (test infrastructure).

Sec. 3.1 with the ideal-gas EOS (Eqs. 15-16): p = (gamma - 1) rho e, c^2 = gamma p / rho,
E = rho |v|^2 / 2 + rho e, gamma = 1.4.  Particles are fixed with volumes w_i; Eq. 18,
divided by the constant w_i, reads with the corrected gradient g_ij = (B_i + B_j)/2 grad W_ij
of Eq. 27 (grad W_ij = grad_i W):

    d rho_i / dt     = -2 sum_j w_j  rho_s (v_s . g_ij)
    d (rho v)_i / dt = -2 sum_j w_j [rho_s v_s (v_s . g_ij) + p_s g_ij]
    d E_i / dt       = -2 sum_j w_j (E_s + p_s) (v_s . g_ij)

where (rho_s, v_s, E_s, p_s) is the state of the pair's Riemann problem at the interface,
from the HLLC solver (Eqs. 20-23) with the dissipation limiter (Eqs. 23-24, eta = 1):

    S_l = u_l - c_l,  S_r = u_r + c_r,  beta = min(eta max((u_l - u_r)/c_bar, 0), 1),
    u*  = (rho_l u_l c_l + rho_r u_r c_r + beta^2 (p_l - p_r)) / (rho_l c_l + rho_r c_r),
    p*  = (p_l + p_r)/2 + beta [rho_r c_r (u* - u_r) + rho_l c_l (u_l - u*)] / 2,
    v*  = u* n + (v_l + v_r)/2 - (u_l + u_r) n / 2,
    rho*_k = rho_k (S_k - u_k)/(S_k - u*),  E*_k = ((S_k - u_k) E_k - p_k u_k + p* u*)/(S_k - u*).

Readings (the paper leaves these open or prints them garbled):
* left = i, right = j, n = -e_ij (from i to j), u_l = v_i . n, u_r = v_j . n,
  c_bar = (c_l + c_r)/2;
* the rho* and E* lines print |v_{l/r}| where the normal velocity u_{l/r} belongs (the
  standard HLLC star state): u is used;
* the limited p* prints a minus between rho_r c_r (u* - u_r) and rho_l c_l (u_l - u*).  The
  unlimited HLLC p* (the mean of Eq. 22's two forms with S_l = u_l - c_l, S_r = u_r + c_r)
  has a plus.  So does the acoustic limit (Eq. 26: p* grows with u_l - u_r), and only the
  plus is unchanged when the sides are swapped, which conservation needs.  The plus is used;
* the interface state is chosen by the wave fan at the interface (it does not move): the
  left state if S_l >= 0 and S_r > 0, the right state if S_r <= 0 and S_l < 0, otherwise a
  star state, the left one if u* > 0, the right one if u* < 0 and their mean at u* = 0.
  The outer states carry their own velocity and pressure, the star states v* and p*.  The
  paper's S_l and S_r can cross for strongly colliding states, and u* = 0 is a tie; this
  choice makes the pair (j, i) see the state (i, j) sees, so that mass, momentum and energy
  are conserved;
* time integration (not stated): forward Euler of (rho, rho v, E) with a fixed dt.
"""
from dataclasses import dataclass

import numpy as np

from .kernels import WENDLAND
from .kgc import kernel_gradients, sym_to_full


@dataclass
class CompressibleParams:
    dom: object          # neighbors.Domain
    dt: float
    gamma: float = 1.4
    eta: float = 1.0


def primitives(rho, mom, E, gamma):
    """(v, p, c) of the conserved variables, Eqs. 15-16."""
    v = mom / rho
    p = (gamma - 1.0) * (E - 0.5 * rho * np.sum(v * v, axis=0))
    c = np.sqrt(gamma * p / rho)
    return v, p, c


def hllc_interface_state(rho_l, vl, p_l, E_l, c_l, rho_r, vr, p_r, E_r, c_r, nrm, eta):
    """The interface state (rho_s, v_s, E_s, p_s) of the limited HLLC solver along nrm."""
    ul = np.sum(vl * nrm, axis=0)
    ur = np.sum(vr * nrm, axis=0)
    sl = ul - c_l
    sr = ur + c_r
    cbar = 0.5 * (c_l + c_r)
    beta = np.minimum(eta * np.maximum((ul - ur) / cbar, 0.0), 1.0)
    zl, zr = rho_l * c_l, rho_r * c_r
    ustar = (zl * ul + zr * ur + beta * beta * (p_l - p_r)) / (zl + zr)
    pstar = 0.5 * (p_l + p_r) + 0.5 * beta * (zr * (ustar - ur) + zl * (ul - ustar))
    vstar = ustar * nrm + 0.5 * (vl + vr) - 0.5 * (ul + ur) * nrm
    with np.errstate(divide="ignore", invalid="ignore"):
        rho_sl = rho_l * (sl - ul) / (sl - ustar)
        rho_sr = rho_r * (sr - ur) / (sr - ustar)
        E_sl = ((sl - ul) * E_l - p_l * ul + pstar * ustar) / (sl - ustar)
        E_sr = ((sr - ur) * E_r - p_r * ur + pstar * ustar) / (sr - ustar)
    # the fan at the interface: the left state when both waves move right, the right state
    # when both move left, else a star state by the sign of u* (their mean at u* = 0, so
    # that the pair (j, i) sees the same state as (i, j))
    left = (sl >= 0.0) & (sr > 0.0)
    right = (sr <= 0.0) & (sl < 0.0)
    rho_st = np.where(ustar > 0.0, rho_sl, np.where(ustar < 0.0, rho_sr, 0.5 * (rho_sl + rho_sr)))
    E_st = np.where(ustar > 0.0, E_sl, np.where(ustar < 0.0, E_sr, 0.5 * (E_sl + E_sr)))
    rho_s = np.where(left, rho_l, np.where(right, rho_r, rho_st))
    E_s = np.where(left, E_l, np.where(right, E_r, E_st))
    p_s = np.where(left, p_l, np.where(right, p_r, pstar))
    v_s = np.where(left, vl, np.where(right, vr, vstar))
    return rho_s, v_s, E_s, p_s


def compressible_rates(pos, vol, rho, mom, E, Bs, row_ptr, col, prm):
    """(d rho/dt (n,), d(rho v)/dt (dim, n), dE/dt (n,)) of Eq. 18 at the given state."""
    dom = prm.dom
    dim = dom.dim
    n = pos.shape[1]
    i, j, rij, r, grad = kernel_gradients(pos, row_ptr, col, dom, WENDLAND)
    B = sym_to_full(Bs, dim)
    g = np.einsum("mab,bm->am", 0.5 * (B[i] + B[j]), grad)
    nrm = -rij / r
    v, p, c = primitives(rho, mom, E, prm.gamma)
    rho_s, v_s, E_s, p_s = hllc_interface_state(rho[i], v[:, i], p[i], E[i], c[i], rho[j], v[:, j], p[j], E[j],
                                                c[j], nrm, prm.eta)
    vg = np.sum(v_s * g, axis=0)
    w = vol[j]
    drho = -2.0 * np.bincount(i, weights=w * rho_s * vg, minlength=n)
    dmom = np.zeros((dim, n))
    for a in range(dim):
        dmom[a] = -2.0 * np.bincount(i, weights=w * (rho_s * v_s[a] * vg + p_s * g[a]), minlength=n)
    dE = -2.0 * np.bincount(i, weights=w * (E_s + p_s) * vg, minlength=n)
    return drho, dmom, dE


def step(pos, vol, rho, mom, E, Bs, row_ptr, col, prm):
    """One forward-Euler step of (rho, rho v, E)."""
    drho, dmom, dE = compressible_rates(pos, vol, rho, mom, E, Bs, row_ptr, col, prm)
    return rho + prm.dt * drho, mom + prm.dt * dmom, E + prm.dt * dE


def run(pos, vol, rho, mom, E, Bs, row_ptr, col, prm, nsteps):
    for _ in range(nsteps):
        rho, mom, E = step(pos, vol, rho, mom, E, Bs, row_ptr, col, prm)
    return rho, mom, E


def exact_riemann(rho_l, u_l, p_l, rho_r, u_r, p_r, xi, gamma=1.4):
    """Exact solution of the 1D Riemann problem of the Euler equations (ideal gas) at
    similarity coordinates xi = x / t: the star pressure from the pressure function by
    Newton's method, then the wave pattern sampled at each xi.  Returns (rho, u, p)."""
    g = gamma
    c_l, c_r = np.sqrt(g * p_l / rho_l), np.sqrt(g * p_r / rho_r)

    def f(pp, rho, p, c):
        if pp > p:        # shock
            A, Bc = 2.0 / ((g + 1.0) * rho), (g - 1.0) / (g + 1.0) * p
            q = np.sqrt(A / (pp + Bc))
            return (pp - p) * q, q * (1.0 - 0.5 * (pp - p) / (pp + Bc))
        # rarefaction
        e = (g - 1.0) / (2.0 * g)
        return 2.0 * c / (g - 1.0) * ((pp / p) ** e - 1.0), (pp / p) ** (-(g + 1.0) / (2.0 * g)) / (rho * c)

    ps = max(1e-12, 0.5 * (p_l + p_r))
    for _ in range(100):
        fl, dl = f(ps, rho_l, p_l, c_l)
        fr, dr = f(ps, rho_r, p_r, c_r)
        nxt = ps - (fl + fr + u_r - u_l) / (dl + dr)
        nxt = max(nxt, 1e-12)
        if abs(nxt - ps) <= 1e-15 * ps:
            ps = nxt
            break
        ps = nxt
    fl, _ = f(ps, rho_l, p_l, c_l)
    fr, _ = f(ps, rho_r, p_r, c_r)
    us = 0.5 * (u_l + u_r) + 0.5 * (fr - fl)
    xi = np.asarray(xi, dtype=np.float64)
    rho = np.empty_like(xi)
    u = np.empty_like(xi)
    p = np.empty_like(xi)
    for k, s in enumerate(xi):
        if s <= us:       # left of the contact
            if ps > p_l:
                sh = u_l - c_l * np.sqrt((g + 1.0) / (2.0 * g) * ps / p_l + (g - 1.0) / (2.0 * g))
                if s <= sh:
                    rho[k], u[k], p[k] = rho_l, u_l, p_l
                else:
                    r = ps / p_l
                    rho[k] = rho_l * (r + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * r + 1.0)
                    u[k], p[k] = us, ps
            else:
                cs = c_l * (ps / p_l) ** ((g - 1.0) / (2.0 * g))
                head, tail = u_l - c_l, us - cs
                if s <= head:
                    rho[k], u[k], p[k] = rho_l, u_l, p_l
                elif s >= tail:
                    rho[k], u[k], p[k] = rho_l * (ps / p_l) ** (1.0 / g), us, ps
                else:
                    uu = 2.0 / (g + 1.0) * (c_l + 0.5 * (g - 1.0) * u_l + s)
                    cc = 2.0 / (g + 1.0) * (c_l + 0.5 * (g - 1.0) * (u_l - s))
                    rho[k] = rho_l * (cc / c_l) ** (2.0 / (g - 1.0))
                    u[k], p[k] = uu, p_l * (cc / c_l) ** (2.0 * g / (g - 1.0))
        else:             # right of the contact
            if ps > p_r:
                sh = u_r + c_r * np.sqrt((g + 1.0) / (2.0 * g) * ps / p_r + (g - 1.0) / (2.0 * g))
                if s >= sh:
                    rho[k], u[k], p[k] = rho_r, u_r, p_r
                else:
                    r = ps / p_r
                    rho[k] = rho_r * (r + (g - 1.0) / (g + 1.0)) / ((g - 1.0) / (g + 1.0) * r + 1.0)
                    u[k], p[k] = us, ps
            else:
                cs = c_r * (ps / p_r) ** ((g - 1.0) / (2.0 * g))
                head, tail = u_r + c_r, us + cs
                if s >= head:
                    rho[k], u[k], p[k] = rho_r, u_r, p_r
                elif s <= tail:
                    rho[k], u[k], p[k] = rho_r * (ps / p_r) ** (1.0 / g), us, ps
                else:
                    uu = 2.0 / (g + 1.0) * (-c_r + 0.5 * (g - 1.0) * u_r + s)
                    cc = 2.0 / (g + 1.0) * (c_r - 0.5 * (g - 1.0) * (u_r - s))
                    rho[k] = rho_r * (cc / c_r) ** (2.0 / (g - 1.0))
                    u[k], p[k] = uu, p_r * (cc / c_r) ** (2.0 * g / (g - 1.0))
    return rho, u, p, ps, us
