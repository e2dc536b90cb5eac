"""Laguerre-Gauss particle relaxation, oracle version (test infrastructure).

Sec. 2.3.2.  Eq. 7 drives particles with a_i = -(2/rho_i) sum_j p0 grad W_ij V_j,
which vanishes at the steady state; the kernel is the Laguerre-Gauss kernel of
Eq. 8 with cut-off 2h.  The paper refers to [zhu2021cad] for how the body
surface is handled and gives no time-step rule.  Readings used here:

* volume V = dp^3, h = 1.3 dp (the smoothing length of the error analysis,
  Sec. 2.3.3), rho = 1, p0 = 1;
* the body is a union of spheres with signed distance
  phi(x) = min_k (|x - c_k| - r_k) (negative inside) and unit normal
  grad phi = (x - c_k*)/|x - c_k*| for the first minimising sphere k*;
* near the surface the part of the kernel support that lies outside the body is
  replaced by its integral over the half-space beyond the tangent plane at
  distance d = max(-phi, 0):  I(d) = integral over {z > d, |r| < 2h} of
  -dW/dr z/|r| dV, applied along grad phi, so that
  a_i = -(2 p0/rho) (sum_j grad W_ij V_j + I(d_i) grad phi_i);
* time step dt = 0.25 sqrt(h / max_i |a_i|) and x_i += a_i dt^2 / 2 (no velocity is
  kept); the displacement h/32 a_i/max|a| is independent of any constant factor in
  a, hence of alpha_d, p0 and rho;
* after the update a particle with phi > -dp/2 is moved back along grad phi to
  phi = -dp/2;
* the neighbour list is rebuilt from the current positions before every step;
* the residual (the "relaxation residue" of Sec. 2.3.3) is
  sqrt(mean over particles with phi < -2h of |h sum_j grad W_ij V_j|^2), evaluated
  with the Laguerre-Gauss kernel (cut-off 2h) and with the truncated Wendland
  kernel (cut-off 1.6h).
"""
import math

import numpy as np

from .kernels import ALPHA_LG, KAPPA_LG, KAPPA_TRUNCATED, LAGUERRE_GAUSS, WENDLAND, kernel_dwdr
from .neighbors import neighbors_cells, pair_geometry, squared_distance


def sdf_spheres(x, spheres):
    """Signed distance to a union of spheres and its gradient.  spheres: (m, 4) rows (c, r)."""
    best = None
    arg = None
    for k in range(spheres.shape[0]):
        dk = np.sqrt(np.sum((x - spheres[k, :3, None]) ** 2, axis=0)) - spheres[k, 3]
        if best is None:
            best = dk
            arg = np.zeros(x.shape[1], dtype=np.int64)
        else:
            upd = dk < best
            best = np.where(upd, dk, best)
            arg = np.where(upd, k, arg)
    c = spheres[arg, :3].T
    rel = x - c
    nrm = np.sqrt(np.sum(rel * rel, axis=0))
    with np.errstate(invalid="ignore", divide="ignore"):
        grad = np.where(nrm > 0.0, rel / nrm, 0.0)
    grad[0] = np.where(nrm > 0.0, grad[0], 1.0)
    return best, grad


def surface_integral_lg(d, h):
    """I(d) = 2 pi int_d^{2h} z (W(z) - W(2h)) dz for the 3D Laguerre-Gauss kernel.

    The inner integral over the plane z = const of -dW/dr z/r reduces to
    2 pi z (W(z) - W(2h)) for a radial kernel; with t = z/h the antiderivative of
    t (1 - t^2/2 + t^4/6) e^{-t^2} is -(1/12) e^{-t^2} (5 - t^2 + t^4)."""
    t0 = np.clip(np.asarray(d, dtype=np.float64) / h, 0.0, 2.0)

    def prim(t):
        return -(1.0 / 12.0) * np.exp(-t * t) * (5.0 - t * t + t ** 4)

    w_cut = (5.0 / 3.0) * math.exp(-4.0)
    val = (prim(2.0) - prim(t0)) - 0.5 * w_cut * (4.0 - t0 * t0)
    return 2.0 * math.pi * ALPHA_LG[3] / h * val


def gradient_sum(pos, vol, row_ptr, col, dom, kind):
    """s_i = sum_j grad W_ij V_j over the listed pairs with d^2 <= (kappa h)^2, shape (dim, n)."""
    n = pos.shape[1]
    i, j, rij, r, = pair_geometry(pos, row_ptr, col, dom)
    within = squared_distance(rij) <= dom.rc2
    dw = np.where(within, kernel_dwdr(kind, r, dom.h, dom.dim, None), 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        scale = np.where(r > 0.0, dw / r, 0.0) * vol[j]
    s = np.zeros((dom.dim, n))
    for a in range(dom.dim):
        s[a] = np.bincount(i, weights=rij[a] * scale, minlength=n)
    return s


def acceleration(pos, vol, row_ptr, col, dom, spheres, p0=1.0, rho=1.0):
    """Eq. 7 with the Laguerre-Gauss kernel and the surface term."""
    s = gradient_sum(pos, vol, row_ptr, col, dom, LAGUERRE_GAUSS)
    phi, gphi = sdf_spheres(pos, spheres)
    surf = surface_integral_lg(np.maximum(-phi, 0.0), dom.h)
    return -(2.0 * p0 / rho) * (s + surf * gphi)


def bound(x, spheres, dp):
    """Move particles with phi > -dp/2 back to phi = -dp/2 along grad phi."""
    phi, gphi = sdf_spheres(x, spheres)
    out = phi > -0.5 * dp
    shift = np.where(out, phi + 0.5 * dp, 0.0)
    return x - shift * gphi


def step(pos, vol, dom, spheres, dp, p0=1.0, rho=1.0, csr=None):
    """One relaxation step from ``pos`` (the CSR is rebuilt unless given)."""
    if csr is None:
        csr = neighbors_cells(pos, dom)
    row_ptr, col = csr
    a = acceleration(pos, vol, row_ptr, col, dom, spheres, p0, rho)
    amax = float(np.max(np.sqrt(np.sum(a * a, axis=0)))) if a.shape[1] else 0.0
    if amax > 0.0:
        dt = 0.25 * math.sqrt(dom.h / amax)
        x = pos + 0.5 * a * (dt * dt)
    else:
        x = pos.copy()
    return bound(x, spheres, dp)


def run(pos, vol, dom, spheres, dp, nsteps, p0=1.0, rho=1.0):
    for _ in range(nsteps):
        pos = step(pos, vol, dom, spheres, dp, p0, rho)
    return pos


def residual(pos, vol, dom, spheres, row_ptr=None, col=None):
    """(R_LG, R_TW, number of interior particles) of the current distribution."""
    dom_lg = dom.with_kappa(KAPPA_LG)
    if row_ptr is None:
        row_ptr, col = neighbors_cells(pos, dom_lg)
    phi, _ = sdf_spheres(pos, spheres)
    interior = phi < -2.0 * dom.h
    m = int(np.sum(interior))
    if m == 0:
        return 0.0, 0.0, 0
    s_lg = gradient_sum(pos, vol, row_ptr, col, dom_lg, LAGUERRE_GAUSS)
    dom_tw = dom.with_kappa(KAPPA_TRUNCATED)
    s_tw = gradient_sum(pos, vol, row_ptr, col, dom_tw, WENDLAND)
    out = []
    for s in (s_lg, s_tw):
        e = dom.h * dom.h * np.sum(s * s, axis=0)
        out.append(math.sqrt(float(np.sum(e[interior])) / m))
    return out[0], out[1], m
