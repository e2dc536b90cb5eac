"""Pins of the oracle's Laguerre-Gauss relaxation (Eqs. 7-8) and of the L2 norm (Eq. 10)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels as K
from oracle import neighbors as N
from oracle import relax as R
from oracle.metrics import l2_error
from paper_2405_05155_gb300 import inputs


def test_l2_norm_eq10():
    ref = np.array([3.0, 4.0])
    assert l2_error(ref, ref * 1.1) == pytest.approx(0.1, abs=1e-15)
    assert l2_error(ref, ref) == 0.0


@pytest.mark.parametrize("d_over_h", [0.0, 0.3, 0.9, 1.5, 1.99, 2.5])
def test_surface_integral_matches_half_space_quadrature(d_over_h):
    # I(d) = int over {z > d, |r| < 2h} of -dW/dr z / r dV, by 2D quadrature in (z, rho)
    h = 0.7
    R2 = 2.0 * h
    d = d_over_h * h

    def integrand(rho, z):
        r = math.hypot(z, rho)
        if r == 0.0 or r > R2:
            return 0.0
        return -float(K.lg_dwdr(r, h, 3, None)) * z / r * 2.0 * math.pi * rho

    if d >= R2:
        ref = 0.0
    else:
        ref, _ = integrate.dblquad(integrand, d, R2, 0.0, lambda z: math.sqrt(max(R2 * R2 - z * z, 0.0)),
                                   epsabs=1e-13, epsrel=1e-11)
    got = float(R.surface_integral_lg(d, h))
    assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref))


def test_sdf_of_sphere_union():
    spheres = np.array([[0.0, 0.0, 0.0, 1.0], [3.0, 0.0, 0.0, 0.5]])
    x = np.array([[0.5, 2.0, 3.0, 3.4], [0.0, 0.0, 0.2, 0.0], [0.0, 0.0, 0.0, 0.0]])
    phi, g = R.sdf_spheres(x, spheres)
    assert np.allclose(phi, [-0.5, 0.5, -0.3, -0.1], atol=1e-15)
    assert np.allclose(g[:, 0], [1.0, 0.0, 0.0]) and np.allclose(g[:, 3], [1.0, 0.0, 0.0])


def _periodic_lattice(n=12, jitter=0.0, seed=0):
    dp = 1.0 / n
    pos = inputs.lattice((n, n, n), dp)
    if jitter:
        pos = np.mod(pos + np.random.default_rng(seed).uniform(-jitter, jitter, pos.shape) * dp, 1.0)
    dom = N.Domain(3, 1.3 * dp, 2.0, [0.0] * 3, [1.0] * 3, [True] * 3)
    far = np.array([[0.5, 0.5, 0.5, 100.0]])   # every particle far inside: no surface term
    return pos, np.full(pos.shape[1], dp ** 3), dom, far, dp


def test_lattice_is_a_zero_of_the_acceleration():
    pos, vol, dom, far, dp = _periodic_lattice()
    rp, col = N.neighbors_cells(pos, dom)
    a = R.acceleration(pos, vol, rp, col, dom, far)
    single = abs(float(K.lg_dwdr(dp, dom.h, 3, None))) * dp ** 3
    assert np.max(np.abs(a)) < 1e-12 * single


def test_total_acceleration_vanishes_and_scale_invariance():
    pos, vol, dom, far, dp = _periodic_lattice(jitter=0.25, seed=3)
    rp, col = N.neighbors_cells(pos, dom)
    a = R.acceleration(pos, vol, rp, col, dom, far)
    assert np.max(np.abs(np.sum(a, axis=1))) < 1e-12 * np.sum(np.abs(a))
    # the step is invariant to a constant factor in the acceleration (p0, rho, alpha_d)
    x1 = R.step(pos, vol, dom, far, dp, p0=1.0)
    x2 = R.step(pos, vol, dom, far, dp, p0=37.0, rho=0.5)
    assert np.max(np.abs(x1 - x2)) < 1e-15 * 10
    # the largest displacement is h/32 (dt = 0.25 sqrt(h/max|a|))
    disp = np.sqrt(np.sum((x1 - pos) ** 2, axis=0))
    assert abs(disp.max() - dom.h / 32.0) < 1e-12


def test_relaxation_lowers_the_residual_and_keeps_particles_inside():
    body = inputs.sphere_body(3, 1.0 / 20.0)
    d = body["domain"]
    dom = N.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])
    pos = body["pos"]
    r0 = R.residual(pos, body["vol"], dom, body["spheres"])
    pos = R.run(pos, body["vol"], dom, body["spheres"], body["dp"], 15)
    r1 = R.residual(pos, body["vol"], dom, body["spheres"])
    assert r1[0] < 0.5 * r0[0]
    phi, _ = R.sdf_spheres(pos, body["spheres"])
    assert np.all(phi <= -0.5 * body["dp"] + 1e-12)
