"""Pins of the oracle's error-analysis pieces (Sec. 2.3.3): the 2D and Wendland surface
integrals of the relaxation, the kernel summation and the weak-form gradient (Eq. 4
with and without the correction matrix of Eq. 9)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import approx as A
from oracle import kernels as K
from oracle import kgc as OK
from oracle import neighbors as N
from oracle import relax as R
from paper_2405_05155_gb300 import inputs


def _dwdr(kind, r, h, dim):
    return float(K.kernel_dwdr(kind, r, h, dim, None))


@pytest.mark.parametrize("kind", [K.LAGUERRE_GAUSS, K.WENDLAND])
@pytest.mark.parametrize("d_over_h", [0.0, 0.4, 1.1, 1.7, 1.99])
def test_surface_integral_2d_matches_half_plane_quadrature(kind, d_over_h):
    # I(d) = int over {z > d, |r| < 2h} of -dW/dr z / r dA, by 2D quadrature in (z, y)
    h = 0.6
    rc = 2.0 * h
    d = d_over_h * h

    def integrand(y, z):
        r = math.hypot(z, y)
        if r == 0.0 or r > rc:
            return 0.0
        return -_dwdr(kind, r, h, 2) * z / r * 2.0

    ref, _ = integrate.dblquad(integrand, d, rc, 0.0, lambda z: math.sqrt(max(rc * rc - z * z, 0.0)),
                               epsabs=1e-13, epsrel=1e-11)
    got = float(R.surface_integral(kind, d, h, 2, 2.0))
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_surface_integral_3d_wendland_and_quadrature_order():
    h = 0.5
    rc = 2.0 * h
    for d in (0.0, 0.3, 0.8):
        ref, _ = integrate.dblquad(
            lambda rho, z: (-_dwdr(K.WENDLAND, math.hypot(z, rho), h, 3) * z / math.hypot(z, rho) * 2 * math.pi * rho
                            if 0.0 < math.hypot(z, rho) <= rc else 0.0),
            d, rc, 0.0, lambda z: math.sqrt(max(rc * rc - z * z, 0.0)), epsabs=1e-13, epsrel=1e-11)
        assert abs(float(R.surface_integral(K.WENDLAND, d, h, 3, 2.0)) - ref) <= 1e-9 * max(1.0, ref)
    # the Gauss-Legendre rule has converged: doubling its order changes nothing
    d = np.linspace(0.0, 2.0 * h, 9)
    a = R.surface_integral(K.LAGUERRE_GAUSS, d, h, 2, 2.0)
    old = R.GL_ORDER
    try:
        R.GL_ORDER = 2 * old
        b = R.surface_integral(K.LAGUERRE_GAUSS, d, h, 2, 2.0)
    finally:
        R.GL_ORDER = old
    assert np.max(np.abs(a - b)) < 1e-13 * np.max(np.abs(b))


def _lattice2d(n=24, periodic=True, h_over_dp=1.3, kappa=2.0):
    dp = 1.0 / n
    pos = inputs.lattice((n, n), dp)
    dom = N.Domain(2, h_over_dp * dp, kappa, [0.0, 0.0], [1.0, 1.0], [periodic, periodic])
    return pos, np.full(pos.shape[1], dp * dp), dom, dp


@pytest.mark.parametrize("kappa,printed", [(2.0, 0.010), (1.6, 0.006)])
def test_kernel_sum_matches_table1_lattice_row(kappa, printed):
    # Table 1, lattice row: L2 of the summation for f = 1 at h = 1.3 dp (SW 0.010, TW 0.006,
    # three decimals); on a full-support lattice every particle has the same sum
    pos, vol, dom, dp = _lattice2d(kappa=kappa)
    rp, col = N.neighbors_cells(pos, dom)
    f = np.ones(pos.shape[1])
    s = A.kernel_sum(pos, vol, f, rp, col, dom)
    assert np.ptp(s) < 1e-13
    err = float(np.sqrt(np.sum((s - f) ** 2) / np.sum(f * f)))
    assert abs(err - printed) < 0.0005 + 1e-12


def test_weak_gradient_brute_force_and_identity():
    # brute force over all pairs on a small jittered box, and the identity that holds for
    # any positions: with B of Eq. 9, sum_j (f_i + f_j) B_i grad W_ij V_j
    # = 2 f_i B_i sum_j grad W_ij V_j + grad f for a linear f
    rng = np.random.default_rng(4)
    n = 7
    dp = 1.0 / n
    pos = inputs.lattice((n, n), dp) + rng.uniform(-0.3, 0.3, (2, n * n)) * dp
    dom = N.Domain(2, 1.3 * dp, 2.0, [-0.2, -0.2], [1.4, 1.4], [False, False])
    vol = np.full(n * n, dp * dp) * rng.uniform(0.9, 1.1, n * n)
    rp, col = N.neighbors_cells(pos, dom)
    a = np.array([0.7, -1.3])
    f = 0.4 + a @ pos
    g = A.weak_gradient(pos, vol, f, rp, col, dom)
    bf = np.zeros_like(g)
    for i in range(n * n):
        for j in range(n * n):
            r = pos[:, i] - pos[:, j]
            d2 = r[0] * r[0] + r[1] * r[1]
            if i == j or d2 > dom.rc2:
                continue
            rr = math.sqrt(d2)
            bf[:, i] += (f[i] + f[j]) * _dwdr(K.WENDLAND, rr, dom.h, 2) / rr * r * vol[j]
    assert np.max(np.abs(g - bf)) < 1e-12 * np.max(np.abs(bf))
    B, fb = OK.kgc(pos, vol, rp, col, dom, K.WENDLAND)
    assert not np.any(fb)
    gB = A.weak_gradient(pos, vol, f, rp, col, dom, B=B)
    s = R.gradient_sum(pos, vol, rp, col, dom, K.WENDLAND)
    Bf = OK.sym_to_full(B, 2)
    pred = 2.0 * f * np.einsum("nab,bn->an", Bf, s) + a[:, None]
    assert np.max(np.abs(gB - pred)) < 1e-11 * np.max(np.abs(pred))


def test_lattice_gradient_with_b_is_exact():
    # a periodic lattice gives sum_j grad W_ij V_j = 0, so the corrected weak form returns
    # the gradient of a linear field exactly at every particle away from the seam
    pos, vol, dom, dp = _lattice2d(n=20, periodic=True, kappa=1.6)
    rp, col = N.neighbors_cells(pos, dom)
    B, fb = OK.kgc(pos, vol, rp, col, dom, K.WENDLAND)
    a = np.array([0.3, 1.1])
    f = a @ pos
    g = A.weak_gradient(pos, vol, f, rp, col, dom, B=B)
    inner = np.all((pos > 0.2) & (pos < 0.8), axis=0)
    assert np.max(np.abs(g[:, inner] - a[:, None])) < 1e-11


@pytest.mark.parametrize("kind", [K.LAGUERRE_GAUSS, K.WENDLAND])
def test_2d_relaxation_lattice_zero_and_surface_balance(kind):
    # (i) a periodic 2D lattice is a zero of Eq. 7 with either kernel; (ii) at a flat wall
    # the surface term cancels the one-sided pair sum of a fine half-plane lattice
    pos, vol, dom, dp = _lattice2d(n=20)
    far = np.array([[0.5, 0.5, 100.0]])
    rp, col = N.neighbors_cells(pos, dom)
    a = R.acceleration(pos, vol, rp, col, dom, far, kind=kind)
    single = abs(_dwdr(kind, dp, dom.h, 2)) * dp * dp
    assert np.max(np.abs(a)) < 1e-12 * single
    # half-plane y < 0 as a circle of huge radius centred far below
    dp = 0.02
    h = 1.3 * dp
    xs = (np.arange(-30, 31)) * dp
    ys = -(np.arange(0, 40) + 0.5) * dp
    X, Y = np.meshgrid(xs, ys)
    pos = np.stack([X.ravel(), Y.ravel()])
    Rb = 1e6
    body = np.array([[0.0, -Rb, Rb]])
    dom = N.Domain(2, h, 2.0, [-1.0, -1.0], [2.0, 1.2], [False, False])
    rp, col = N.neighbors_cells(pos, dom)
    vol = np.full(pos.shape[1], dp * dp)
    acc = R.acceleration(pos, vol, rp, col, dom, body, kind=kind)
    probe = (np.abs(pos[0]) < 1e-9) & (pos[1] > -3.0 * h)
    scale = float(np.max(np.abs(R.surface_integral(kind, 0.0, h, 2, 2.0)))) * 2.0
    assert np.max(np.abs(acc[:, probe])) < 0.05 * scale
