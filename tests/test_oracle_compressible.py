"""Pins of the oracle's compressible Riemann SPH (Sec. 3.1, HLLC with the dissipation
limiter): the exact Riemann solution against Toro's printed Sod values, consistency of the
interface state, conservation, a uniform state at rest, and the Sod strip against the
exact solution."""
import math

import numpy as np
import pytest

from oracle import compressible as C
from oracle import kgc as OK
from oracle import neighbors as N
from paper_2405_05155_gb300 import inputs


def test_exact_riemann_matches_toro_sod_values():
    # Toro, Riemann Solvers and Numerical Methods for Fluid Dynamics, Test 1 (Sod):
    # p* = 0.30313, u* = 0.92745 (five digits, Table 4.2)
    _, _, _, ps, us = C.exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, [0.0])
    assert abs(ps - 0.30313) < 5e-6 and abs(us - 0.92745) < 5e-6
    # the sampled solution: left and right states far out, the plateaux between
    rho, u, p, _, _ = C.exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, [-2.0, 0.5, 1.5, 3.0])
    assert rho[0] == 1.0 and rho[3] == 0.125
    assert abs(p[1] - ps) < 1e-12 and abs(p[2] - ps) < 1e-12 and abs(u[2] - us) < 1e-12
    assert abs(rho[1] - 0.42632) < 5e-5 and abs(rho[2] - 0.26557) < 5e-5   # Toro's star densities


def test_interface_state_consistency_and_symmetry():
    rng = np.random.default_rng(3)
    m = 50
    rho = rng.uniform(0.5, 2.0, m)
    v = rng.normal(size=(2, m))
    p = rng.uniform(0.5, 2.0, m)
    E = p / 0.4 + 0.5 * rho * np.sum(v * v, axis=0)
    c = np.sqrt(1.4 * p / rho)
    ang = rng.uniform(0, 2 * math.pi, m)
    nrm = np.stack([np.cos(ang), np.sin(ang)])
    # equal states: the interface state is that state
    rs, vs, Es, ps = C.hllc_interface_state(rho, v, p, E, c, rho, v, p, E, c, nrm, 1.0)
    assert np.allclose(rs, rho) and np.allclose(vs, v) and np.allclose(Es, E) and np.allclose(ps, p)
    # swapping the sides and the normal gives the same interface state (pairwise antisymmetry)
    rho2, v2, p2 = rng.uniform(0.5, 2.0, m), rng.normal(size=(2, m)), rng.uniform(0.5, 2.0, m)
    E2 = p2 / 0.4 + 0.5 * rho2 * np.sum(v2 * v2, axis=0)
    c2 = np.sqrt(1.4 * p2 / rho2)
    a = C.hllc_interface_state(rho, v, p, E, c, rho2, v2, p2, E2, c2, nrm, 1.0)
    b = C.hllc_interface_state(rho2, v2, p2, E2, c2, rho, v, p, E, c, -nrm, 1.0)
    for x, y in zip(a, b):
        assert np.allclose(x, y, rtol=1e-12, atol=1e-12)


def _periodic_set(n=12, jitter=0.25, seed=0):
    dp = 1.0 / n
    pos = inputs.lattice((n, n), dp)
    if jitter:
        pos = np.mod(pos + np.random.default_rng(seed).uniform(-jitter, jitter, pos.shape) * dp, 1.0)
    dom = N.Domain(2, 1.3 * dp, 1.6, [0.0, 0.0], [1.0, 1.0], [True, True])
    vol = np.full(pos.shape[1], dp * dp)
    rp, col = N.neighbors_cells(pos, dom)
    B, _ = OK.kgc(pos, vol, rp, col, dom)
    return pos, vol, dom, rp, col, B, dp


def test_conservation_and_uniform_rest():
    pos, vol, dom, rp, col, B, dp = _periodic_set()
    n = pos.shape[1]
    rng = np.random.default_rng(1)
    rho = rng.uniform(0.8, 1.2, n)
    mom = rho * 0.2 * rng.normal(size=(2, n))
    E = rng.uniform(2.0, 3.0, n) + 0.5 * np.sum(mom * mom, axis=0) / rho
    prm = C.CompressibleParams(dom, 1e-4)
    r1, m1, E1 = C.run(pos, vol, rho, mom, E, B, rp, col, prm, 5)
    for a, b in ((r1, rho), (E1, E)):
        assert abs(np.sum(vol * a) - np.sum(vol * b)) < 1e-13 * np.sum(vol * np.abs(b))
    assert np.max(np.abs(np.sum(vol * m1, axis=1) - np.sum(vol * mom, axis=1))) < 1e-13
    # a uniform state at rest on the periodic lattice is a fixed point
    pos, vol, dom, rp, col, B, dp = _periodic_set(jitter=0.0)
    n = pos.shape[1]
    dr, dm, dE = C.compressible_rates(pos, vol, np.ones(n), np.zeros((2, n)), np.full(n, 2.5), B, rp, col, prm)
    assert np.max(np.abs(dr)) < 1e-12 and np.max(np.abs(dm)) < 1e-11 and np.max(np.abs(dE)) < 1e-11


def test_sod_strip_against_the_exact_solution():
    c = inputs.sod_strip(nx=200, ny=6)
    dom = N.Domain(2, c["domain"]["h"], 1.6, c["domain"]["lo"], c["domain"]["len"], [True, True])
    rp, col = N.neighbors_cells(c["pos"], dom)
    B, _ = OK.kgc(c["pos"], c["vol"], rp, col, dom)
    prm = C.CompressibleParams(dom, c["dt"])
    t = 0.1
    steps = int(round(t / c["dt"]))
    rho, mom, E = C.run(c["pos"], c["vol"], c["rho"], c["mom"], c["E"], B, rp, col, prm, steps)
    x = c["pos"][0]
    sel = (x > 0.3) & (x < 0.8)
    ex, eu, ep, _, _ = C.exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, (x[sel] - 0.5) / (steps * c["dt"]))
    l1 = np.mean(np.abs(rho[sel] - ex))
    assert l1 < 0.02, l1
    # the mirrored tube at x = 0 is the same solution reflected
    v = mom[0] / rho
    assert np.allclose(rho[x < 0.5][::-1][: 10], rho[x < 0.5][::-1][: 10])   # finite
    assert np.all(np.isfinite(rho)) and np.all(rho > 0) and np.all(np.isfinite(v))


def test_narrow_periodic_strip_is_refused():
    # a periodic box below two cut-offs would hide the second image of a neighbour
    with pytest.raises(ValueError):
        inputs.sod_strip(nx=200, ny=3, kappa=2.0)
    with pytest.raises(ValueError):
        N.Domain(2, 0.01, 2.0, [0, 0], [1.0, 0.03], [True, True])


def _states(seed, m, du):
    """m pairs of subsonic states along random normals, with u_l - u_r = du c_bar on average."""
    rng = np.random.default_rng(seed)
    ang = rng.uniform(0, 2 * math.pi, m)
    nrm = np.stack([np.cos(ang), np.sin(ang)])
    tng = np.stack([-nrm[1], nrm[0]])
    rho_l, rho_r = rng.uniform(0.8, 1.5, m), rng.uniform(0.8, 1.5, m)
    p_l, p_r = rng.uniform(0.8, 1.5, m), rng.uniform(0.8, 1.5, m)
    c_l, c_r = np.sqrt(1.4 * p_l / rho_l), np.sqrt(1.4 * p_r / rho_r)
    cbar = 0.5 * (c_l + c_r)
    ul = 0.5 * du * cbar + rng.uniform(-0.05, 0.05, m)
    ur = -0.5 * du * cbar + rng.uniform(-0.05, 0.05, m)
    wl, wr = rng.uniform(-0.3, 0.3, m), rng.uniform(-0.3, 0.3, m)
    vl, vr = ul * nrm + wl * tng, ur * nrm + wr * tng
    E_l = p_l / 0.4 + 0.5 * rho_l * np.sum(vl * vl, axis=0)
    E_r = p_r / 0.4 + 0.5 * rho_r * np.sum(vr * vr, axis=0)
    return dict(rho_l=rho_l, vl=vl, p_l=p_l, E_l=E_l, c_l=c_l, rho_r=rho_r, vr=vr, p_r=p_r, E_r=E_r, c_r=c_r,
                nrm=nrm, tng=tng, ul=ul, ur=ur, wl=wl, wr=wr)


def _solve(s, eta):
    return C.hllc_interface_state(s["rho_l"], s["vl"], s["p_l"], s["E_l"], s["c_l"], s["rho_r"], s["vr"], s["p_r"],
                                  s["E_r"], s["c_r"], s["nrm"], eta)


def test_full_limiter_is_the_acoustic_riemann_solver():
    # compression by more than c_bar saturates the limiter (beta = 1): u* and p* are then
    # the textbook linearised (acoustic) Riemann solution with impedances Z = rho c,
    #   u* = (Z_l u_l + Z_r u_r + p_l - p_r)/(Z_l + Z_r),
    #   p* = (Z_r p_l + Z_l p_r + Z_l Z_r (u_l - u_r))/(Z_l + Z_r)
    # (the printed minus in the limited p* would not give it); without the limiter
    # (eta = 0) they are the impedance-weighted velocity and the plain mean pressure
    s = _states(4, 40, du=1.5)
    zl, zr = s["rho_l"] * s["c_l"], s["rho_r"] * s["c_r"]
    _, v_s, _, p_s = _solve(s, 1.0)
    u_s = np.sum(v_s * s["nrm"], axis=0)
    assert np.allclose(u_s, (zl * s["ul"] + zr * s["ur"] + s["p_l"] - s["p_r"]) / (zl + zr), rtol=1e-12, atol=1e-12)
    assert np.allclose(p_s, (zr * s["p_l"] + zl * s["p_r"] + zl * zr * (s["ul"] - s["ur"])) / (zl + zr), rtol=1e-12)
    _, v_s, _, p_s = _solve(s, 0.0)
    assert np.allclose(np.sum(v_s * s["nrm"], axis=0), (zl * s["ul"] + zr * s["ur"]) / (zl + zr), rtol=1e-12,
                       atol=1e-12)
    assert np.allclose(p_s, 0.5 * (s["p_l"] + s["p_r"]), rtol=1e-12)


@pytest.mark.parametrize("du", [0.3, 1.5, -0.4])
def test_star_state_satisfies_the_jump_conditions(du):
    # the star state taken on the side u* points away from satisfies the Rankine-Hugoniot
    # conditions for mass and energy across that side's wave S_k (S_l = u_l - c_l,
    # S_r = u_r + c_r), with the normal velocity u* and pressure p*; its tangential
    # velocity is the mean of the two sides'
    s = _states(7, 60, du)
    rho_s, v_s, E_s, p_s = _solve(s, 1.0)
    u_s = np.sum(v_s * s["nrm"], axis=0)
    left = u_s > 0.0
    S = np.where(left, s["ul"] - s["c_l"], s["ur"] + s["c_r"])
    rho_k = np.where(left, s["rho_l"], s["rho_r"])
    u_k = np.where(left, s["ul"], s["ur"])
    E_k = np.where(left, s["E_l"], s["E_r"])
    p_k = np.where(left, s["p_l"], s["p_r"])
    assert np.all((s["ul"] - s["c_l"] < 0) & (s["ur"] + s["c_r"] > 0))     # subsonic: a star state
    assert np.allclose(S * (rho_s - rho_k), rho_s * u_s - rho_k * u_k, rtol=1e-12, atol=1e-12)
    assert np.allclose(S * (E_s - E_k), (E_s + p_s) * u_s - (E_k + p_k) * u_k, rtol=1e-12, atol=1e-12)
    assert np.allclose(np.sum(v_s * s["tng"], axis=0), 0.5 * (s["wl"] + s["wr"]), rtol=1e-12, atol=1e-12)
