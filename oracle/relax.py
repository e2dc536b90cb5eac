"""Laguerre-Gauss particle relaxation, oracle version (test infrastructure).

Sec. 2.3.2.  Eq. 7 drives particles with a_i = -(2/rho_i) sum_j p0 grad W_ij V_j,
which vanishes at the steady state; the kernel is the Laguerre-Gauss kernel of
Eq. 8 with cut-off 2h.  The paper refers to [zhu2021cad] for how the body
surface is handled and gives no time-step rule.  Readings used here:

* volume V = dp^d, h = 1.3 dp (the smoothing length of the error analysis,
  Sec. 2.3.3), rho = 1, p0 = 1; 2D bodies are unions of circles;
* the Wendland-relaxed distributions of Sec. 2.3.3 use the same step with the
  standard Wendland kernel (cut-off 2h) in place of the Laguerre-Gauss kernel;
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
    """Signed distance to a union of spheres (circles in 2D) and its gradient.
    spheres: (m, dim + 1) rows (centre, radius)."""
    dim = x.shape[0]
    best = None
    arg = None
    for k in range(spheres.shape[0]):
        dk = np.sqrt(np.sum((x - spheres[k, :dim, None]) ** 2, axis=0)) - spheres[k, dim]
        if best is None:
            best = dk
            arg = np.zeros(x.shape[1], dtype=np.int64)
        else:
            upd = dk < best
            best = np.where(upd, dk, best)
            arg = np.where(upd, k, arg)
    c = spheres[arg, :dim].T
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


# Gauss-Legendre order of the surface integrals evaluated by quadrature.
GL_ORDER = 48


def surface_integral(kind, d, h, dim, kappa):
    """I(d): the integral of -dW/dr z/|r| over the part of the support beyond a plane
    at distance d (z measured from the particle along the normal), for a radial
    kernel cut at kappa h.  Integrating over lines (2D) or planes (3D) of constant z
    first:
      2D: I(d) = 2 int_0^Y (W(sqrt(d^2 + y^2)) - W(kappa h)) dy,  Y = sqrt((kappa h)^2 - d^2);
      3D: I(d) = 2 pi int_d^{kappa h} z (W(z) - W(kappa h)) dz.
    The 3D Laguerre-Gauss case uses the closed form of surface_integral_lg; the others
    a Gauss-Legendre rule of GL_ORDER nodes (the integrands are smooth)."""
    d = np.clip(np.asarray(d, dtype=np.float64), 0.0, kappa * h)
    if dim == 3 and kind == LAGUERRE_GAUSS and kappa == KAPPA_LG:
        return surface_integral_lg(d, h)
    from .kernels import kernel_w
    rc = kappa * h
    w_cut = float(kernel_w(kind, rc, h, dim, None))
    x, w = np.polynomial.legendre.leggauss(GL_ORDER)
    u = 0.5 * (x + 1.0)                      # nodes on [0, 1]
    wt = 0.5 * w
    flat = d.reshape(-1)
    out = np.empty_like(flat)
    for k, dk in enumerate(flat):
        if dim == 2:
            Y = math.sqrt(max(rc * rc - dk * dk, 0.0))
            y = Y * u
            f = kernel_w(kind, np.sqrt(dk * dk + y * y), h, 2, None) - w_cut
            out[k] = 2.0 * Y * float(np.sum(wt * f))
        else:
            z = dk + (rc - dk) * u
            f = z * (kernel_w(kind, z, h, 3, None) - w_cut)
            out[k] = 2.0 * math.pi * (rc - dk) * float(np.sum(wt * f))
    return out.reshape(d.shape)


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


def acceleration(pos, vol, row_ptr, col, dom, spheres, p0=1.0, rho=1.0, kind=LAGUERRE_GAUSS):
    """Eq. 7 with the surface term; the Laguerre-Gauss kernel (Eq. 8) or, for the
    Wendland-relaxed distributions of Sec. 2.3.3, the standard Wendland kernel, each
    cut at dom.kappa h."""
    s = gradient_sum(pos, vol, row_ptr, col, dom, kind)
    phi, gphi = sdf_spheres(pos, spheres)
    surf = surface_integral(kind, np.maximum(-phi, 0.0), dom.h, dom.dim, dom.kappa)
    return -(2.0 * p0 / rho) * (s + surf * gphi)


def bound(x, spheres, dp):
    """Move particles with phi > -dp/2 back to phi = -dp/2 along grad phi."""
    phi, gphi = sdf_spheres(x, spheres)
    out = phi > -0.5 * dp
    shift = np.where(out, phi + 0.5 * dp, 0.0)
    return x - shift * gphi


def step(pos, vol, dom, spheres, dp, p0=1.0, rho=1.0, csr=None, kind=LAGUERRE_GAUSS):
    """One relaxation step from ``pos`` (the CSR is rebuilt unless given)."""
    if csr is None:
        csr = neighbors_cells(pos, dom)
    row_ptr, col = csr
    a = acceleration(pos, vol, row_ptr, col, dom, spheres, p0, rho, kind)
    amax = float(np.max(np.sqrt(np.sum(a * a, axis=0)))) if a.shape[1] else 0.0
    if amax > 0.0:
        dt = 0.25 * math.sqrt(dom.h / amax)
        x = pos + 0.5 * a * (dt * dt)
    else:
        x = pos.copy()
    return bound(x, spheres, dp)


def run(pos, vol, dom, spheres, dp, nsteps, p0=1.0, rho=1.0, kind=LAGUERRE_GAUSS):
    for _ in range(nsteps):
        pos = step(pos, vol, dom, spheres, dp, p0, rho, kind=kind)
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
