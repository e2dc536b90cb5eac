"""Pins of the oracle's total-Lagrangian solid update (Eqs. 28-31)."""
import math

import numpy as np
import pytest

from oracle import kgc as G
from oracle import neighbors as N
from oracle import tlsph as T
from paper_2405_05155_gb300 import inputs


def _plate(dp=0.005, kappa=1.6):
    c = inputs.plate(dp=dp, kappa=kappa)
    d = c["domain"]
    dom = N.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])
    rp, col = N.neighbors_cells(c["r0"], dom)
    B0, fb = G.kgc(c["r0"], c["vol"], rp, col, dom)
    return c, dom, rp, col, B0, fb


def test_lame_parameters():
    lam, G_ = T.lame(2.0e6, 0.3975)
    assert abs(lam - 2.0e6 * 0.3975 / (1.3975 * 0.205)) < 1e-6
    assert abs(G_ - 2.0e6 / 2.795) < 1e-9
    # consistency with the bulk modulus K = lambda + 2G/3 = E / (3 (1 - 2 nu))
    assert abs(lam + 2.0 * G_ / 3.0 - 2.0e6 / (3.0 * (1.0 - 2.0 * 0.3975))) < 1e-6


def test_stress_uniaxial_hand_values():
    s = 1.1
    F = np.diag([s, 1.0, 1.0])[None]
    lam, G_ = 3.0, 2.0
    # SVK: E11 = (s^2 - 1)/2, S11 = (lam + 2G) E11, S22 = S33 = lam E11, P11 = s S11
    E11 = 0.5 * (s * s - 1.0)
    S = T.pk2_svk(F, lam, G_)[0]
    assert np.allclose(np.diag(S), [(lam + 2 * G_) * E11, lam * E11, lam * E11], atol=1e-14)
    P = T.first_piola(F, T.pk2_svk(F, lam, G_))[0]
    assert abs(P[0, 0] - s * (lam + 2 * G_) * E11) < 1e-14
    # neo-Hookean: S11 = G (1 - 1/s^2) + lam ln(s)/s^2, S22 = S33 = lam ln s
    S = T.pk2_neo_hookean(F, lam, G_)[0]
    assert np.allclose(np.diag(S), [G_ * (1 - 1 / s ** 2) + lam * math.log(s) / s ** 2,
                                    lam * math.log(s), lam * math.log(s)], atol=1e-14)
    assert np.max(np.abs(S - np.diag(np.diag(S)))) == 0.0


def test_linear_velocity_field_gives_exact_rate():
    # Eq. 31 with B0 reproduces dF/dt = L for v = L r + c at every particle with a regular A
    c, dom, rp, col, B0, fb = _plate()
    rng = np.random.default_rng(3)
    L = rng.normal(size=(3, 3))
    v = L @ c["r0"] + rng.normal(size=(3, 1))
    Fdot = T.deformation_rate(c["r0"], c["vol"], v, B0, rp, col, dom)
    ok = fb == 0
    assert ok.sum() > 0.99 * ok.size
    assert np.max(np.abs(Fdot[ok] - L[None])) < 1e-9 * np.max(np.abs(L))


@pytest.mark.parametrize("law", [T.SVK, T.NEO_HOOKEAN])
def test_undeformed_state_is_stress_free_and_momentum_conserved(law):
    c, dom, rp, col, B0, fb = _plate()
    n = c["r0"].shape[1]
    prm = T.TLParams(dom, c["dt"], c["rho0"], c["lam"], c["G"], law)
    F = np.tile(np.eye(3), (n, 1, 1))
    M = T.stress_matrix(F, B0, prm)
    assert np.max(np.abs(M)) < 1e-9
    a = T.momentum_rate(c["r0"], c["vol"], M, rp, col, dom, prm.rho0)
    assert np.max(np.abs(a)) < 1e-9
    # a random deformation: total force sum_i V0 rho0 a_i vanishes (pairwise antisymmetry)
    rng = np.random.default_rng(1)
    F = F + 0.01 * rng.normal(size=F.shape)
    M = T.stress_matrix(F, B0, prm)
    a = T.momentum_rate(c["r0"], c["vol"], M, rp, col, dom, prm.rho0)
    tot = np.sum(c["vol"] * prm.rho0 * a, axis=1)
    scale = np.sum(c["vol"] * prm.rho0 * np.abs(a))
    assert np.max(np.abs(tot)) < 1e-12 * scale


def test_energy_is_nearly_conserved():
    c, dom, rp, col, B0, fb = _plate(dp=0.01)
    n = c["r0"].shape[1]
    prm = T.TLParams(dom, c["dt"], c["rho0"], c["lam"], c["G"], T.NEO_HOOKEAN)
    F = np.tile(np.eye(3), (n, 1, 1))
    x, v = c["r0"].copy(), c["v"].copy()
    e0 = sum(T.energies(c["r0"], c["vol"], v, F, prm))
    x, v, F = T.run(c["r0"], c["vol"], B0, c["fixed"], x, v, F, rp, col, prm, 100)
    ke, pe = T.energies(c["r0"], c["vol"], v, F, prm)
    assert pe > 0.01 * e0          # energy moved into the strain field
    assert abs(ke + pe - e0) < 0.01 * e0
    assert np.all(v[:, c["fixed"] == 1] == 0.0)


def test_column_initial_fields():
    # Sec. 5 columns: the twisting field is a rotation of each horizontal slice about the
    # column axis at rate 105 sin(pi y / 12); the bending field is uniform; the base is clamped
    from paper_2405_05155_gb300 import inputs
    c = inputs.column("twisting", 6)
    x, y, z = c["r0"]
    vx, vy, vz = c["v"]
    free = c["fixed"] == 0
    dx, dz = x - 0.5, z - 0.5
    assert np.all(c["v"][:, ~free] == 0.0)
    assert np.max(np.abs((vx * dx + vz * dz)[free])) < 1e-12
    rate = 105.0 * np.sin(np.pi * y / 12.0)
    assert np.allclose(np.hypot(vx, vz)[free], (np.abs(rate) * np.hypot(dx, dz))[free])
    assert np.all(vy == 0.0) and c["nu"] == 0.499
    b = inputs.column("bending", 6)
    free = b["fixed"] == 0
    assert np.allclose(b["v"][:, free], np.array([[10 * np.sqrt(3) / 2], [5.0], [0.0]]))
    assert b["nu"] == 0.45 and np.isclose(b["G"], 17e6 / 2.9)
