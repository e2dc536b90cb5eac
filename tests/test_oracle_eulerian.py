"""Pins of the oracle's Eulerian WCSPH update (Eqs. 18, 22, 25-27)."""
import math

import numpy as np
import pytest

from oracle import eulerian as E
from oracle import kgc as G
from oracle import neighbors as N
from oracle.metrics import l2_error
from paper_2405_05155_gb300 import inputs


def _dom(d):
    return N.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])


def test_riemann_special_cases():
    rng = np.random.default_rng(0)
    u = rng.normal(size=50)
    p = rng.normal(size=50)
    rho = 1.0 + 0.01 * rng.normal(size=50)
    c = 10.0
    # equal states: the star state is the state itself
    us, ps = E.acoustic_star_state(u, u, p, p, rho, c, 15.0)
    assert np.allclose(us, u, atol=1e-15, rtol=0) and np.allclose(ps, p, atol=1e-15, rtol=0)
    # expansion (u_l < u_r): the limiter switches dissipation off (beta = 0)
    us, ps = E.acoustic_star_state(u - 1.0, u + 1.0, p, 2 * p, rho, c, 15.0)
    assert np.allclose(us, u, atol=1e-14) and np.allclose(ps, 1.5 * p, atol=1e-14)
    # strong compression (beta = 1): the plain linearised solver of Eq. 22
    ul, ur = u + 2.0, u - 2.0
    us, ps = E.acoustic_star_state(ul, ur, p, 2 * p, rho, c, 15.0)
    assert np.allclose(us, 0.5 * (ul + ur) + 0.5 * (p - 2 * p) / (rho * c), atol=1e-14)
    assert np.allclose(ps, 0.5 * (p + 2 * p) + 0.5 * rho * c * (ul - ur), atol=1e-13)
    # weak compression: beta = 15 (u_l - u_r)/c
    du = 0.01
    us, ps = E.acoustic_star_state(np.array([du]), np.array([0.0]), np.array([1.0]), np.array([0.0]),
                                   np.array([1.0]), c, 15.0)
    beta = 15.0 * du / c
    assert abs(us[0] - (0.5 * du + 0.5 * beta * beta / c)) < 1e-15
    assert abs(ps[0] - (0.5 + 0.5 * beta * c * du)) < 1e-15


def _random_state(dim, nx, kappa, seed, mu=0.01):
    case = inputs.tgv2d(nx=nx, kappa=kappa) if dim == 2 else inputs.tgv3d(n=nx, kappa=kappa)
    dom = _dom(case["domain"])
    rng = np.random.default_rng(seed)
    dp = case["dp"]
    pos = np.mod(case["pos"] + rng.uniform(-0.2, 0.2, size=case["pos"].shape) * dp, dom.len[0])
    rp, col = N.neighbors_cells(pos, dom)
    Bs, fb = G.kgc(pos, case["vol"], rp, col, dom)
    drho = 0.01 * rng.normal(size=pos.shape[1])
    v = rng.normal(size=pos.shape)
    prm = E.EulerianParams(dom, case["dt"], 1.0, 10.0, mu)
    return pos, case["vol"], drho, v, Bs, rp, col, prm


@pytest.mark.parametrize("dim", [2, 3])
def test_pairwise_antisymmetry_conserves_mass_and_momentum(dim):
    pos, vol, drho, v, Bs, rp, col, prm = _random_state(dim, 24 if dim == 2 else 10, 1.6, 4)
    drho_dt, dmom_dt = E.eulerian_rates(pos, vol, drho, v, Bs, rp, col, prm)
    scale_m = np.sum(vol * np.abs(drho_dt))
    scale_p = np.sum(vol * np.abs(dmom_dt))
    assert abs(np.sum(vol * drho_dt)) < 1e-12 * scale_m
    assert np.max(np.abs(np.sum(vol * dmom_dt, axis=1))) < 1e-12 * scale_p
    # and the rates are not trivially zero
    assert scale_m > 0.0 and scale_p > 0.0


@pytest.mark.parametrize("dim", [2, 3])
def test_uniform_state_is_a_fixed_point(dim):
    case = inputs.tgv2d(nx=20) if dim == 2 else inputs.tgv3d(n=10)
    dom = _dom(case["domain"])
    pos = case["pos"]
    rp, col = N.neighbors_cells(pos, dom)
    Bs, _ = G.kgc(pos, case["vol"], rp, col, dom)
    prm = E.EulerianParams(dom, case["dt"], 1.0, 10.0, 0.05)
    n = pos.shape[1]
    for vel in (0.0, 0.3):
        v = np.zeros((dim, n))
        v[0] = vel
        drho = np.full(n, 0.004)
        drho_dt, dmom_dt = E.eulerian_rates(pos, case["vol"], drho, v, Bs, rp, col, prm)
        assert np.max(np.abs(drho_dt)) < 1e-11
        assert np.max(np.abs(dmom_dt)) < 1e-10


def test_viscous_term_is_a_laplacian():
    # shear flow u = sin(2 pi y) at zero pressure: d(rho u)/dt ~ mu u'' = -mu (2 pi)^2 sin(2 pi y)
    # (the Riemann part vanishes: u_l = u_r along every pair normal only in the mean)
    case = inputs.tgv2d(nx=40)
    dom = _dom(case["domain"]).with_kappa(2.0)
    pos = case["pos"]
    rp, col = N.neighbors_cells(pos, dom)
    Bs, _ = G.kgc(pos, case["vol"], rp, col, dom)
    n = pos.shape[1]
    v = np.zeros((2, n))
    v[0] = np.sin(2 * math.pi * pos[1])
    prm_v = E.EulerianParams(dom, case["dt"], 1.0, 10.0, 0.01)
    prm_0 = E.EulerianParams(dom, case["dt"], 1.0, 10.0, 0.0)
    _, with_mu = E.eulerian_rates(pos, case["vol"], np.zeros(n), v, Bs, rp, col, prm_v)
    _, without = E.eulerian_rates(pos, case["vol"], np.zeros(n), v, Bs, rp, col, prm_0)
    visc = with_mu[0] - without[0]
    exact = -0.01 * (2 * math.pi) ** 2 * v[0]
    assert l2_error(exact, visc) < 0.05


def test_taylor_green_decay_200_steps():
    # 2D TGV of the plain-method workload: 50x50, h = 1.3 dp, kappa = 1.6, Re = 100, 200 steps;
    # the velocity decays as exp(-8 pi^2 t / Re) (closed form).
    case = inputs.tgv2d(nx=50, kappa=1.6)
    dom = _dom(case["domain"])
    pos = case["pos"]
    rp, col = N.neighbors_cells(pos, dom)
    Bs, fb = G.kgc(pos, case["vol"], rp, col, dom)
    prm = E.EulerianParams(dom, case["dt"], case["rho0"], case["c0"], case["mu"])
    drho = case["p"] / case["c0"] ** 2
    drho1, v1 = E.run(pos, case["vol"], drho, case["v"], Bs, rp, col, prm, 200)
    t = 200 * case["dt"]
    exact = inputs.tgv2d_exact_velocity(pos, case["U"], case["nu"], t)
    ratio = np.sqrt(np.mean(v1 ** 2)) / np.sqrt(np.mean(case["v"] ** 2))
    assert abs(ratio / math.exp(-case["decay_rate"] * t) - 1.0) < 0.03
    assert l2_error(exact, v1) < 0.03
    # the pressure keeps its closed-form pattern p ~ cos 4 pi x + cos 4 pi y
    p1 = case["c0"] ** 2 * drho1
    assert np.corrcoef(p1, case["p"])[0, 1] > 0.95


def test_two_pass_and_fused_agree_to_first_order():
    pos, vol, drho, v, Bs, rp, col, prm = _random_state(2, 20, 1.6, 8)
    diffs = []
    for dt in (2e-5, 1e-5):
        prm.dt = dt
        a = E.step_two_pass(pos, vol, drho, v, Bs, rp, col, prm)
        b = E.step_fused(pos, vol, drho, v, Bs, rp, col, prm)
        diffs.append(max(np.max(np.abs(a[1] - b[1])), np.max(np.abs(a[0] - b[0]))))
    # both are consistent one-step integrators: they differ by O(dt^2)
    assert 3.5 < diffs[0] / diffs[1] < 4.5


def test_double_shear_layer_initial_field():
    # the closed form of the initial velocity: u_x = +-1 far from the layers, 0 at y = 1/4
    # and 3/4, tanh profile of thickness 1/30; u_y = 0.05 sin(2 pi x); divergence free
    from paper_2405_05155_gb300 import inputs
    c = inputs.double_shear_layer(nx=64)
    x, y = c["pos"]
    ux, uy = c["v"]
    # +1 between the layers (y near 1/2), -1 outside them (y near 0 or 1)
    assert np.allclose(ux[np.abs(y - 0.5) < 0.1], 1.0, atol=1e-3)
    assert np.allclose(ux[(y < 0.1) | (y > 0.9)], -1.0, atol=1e-3)
    # odd about each layer's centre line: u_x(1/4 + s) = -u_x(1/4 - s) on the lattice rows
    rows = np.unique(np.round(y, 12))
    below = rows[rows < 0.25]
    for yb in below[-3:]:
        ya = 0.5 - yb
        assert np.allclose(ux[np.isclose(y, yb)], -ux[np.isclose(y, ya)])
    assert np.allclose(ux, np.where(y <= 0.5, np.tanh((y - 0.25) * 30.0), np.tanh((0.75 - y) * 30.0)))
    assert np.allclose(uy, 0.05 * np.sin(2.0 * np.pi * x))
    assert c["mu"] == 0.0 and c["dt"] == 0.25 * c["domain"]["h"] / 11.0
