"""GPU parity of the total-Lagrangian solid path (a7-a9) against the float64 oracle."""
import numpy as np
import pytest

from helpers import cuda, host, odom, rel_l2, rel_max, sample_rows, sorted_by_cells
from oracle import kgc as OK
from oracle import tlsph as OT
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _setup(ctx, dp=0.005, kappa=1.6, law=OT.NEO_HOOKEAN):
    c = inputs.plate(dp=dp, kappa=kappa)
    d = c["domain"]
    r0, order = sorted_by_cells(c["r0"], d)
    v = c["v"][:, order]
    fixed = c["fixed"][order]
    vol = c["vol"][order]
    rp, col = api.build_neighbors(ctx, d, cuda(r0))
    B0, fb, _ = api.kgc(ctx, d, cuda(r0), cuda(vol), rp, col)
    prm = OT.TLParams(odom(d), c["dt"], c["rho0"], c["lam"], c["G"], law)
    return dict(c=c, d=d, r0=r0, v=v, fixed=fixed, vol=vol, rp=rp, col=col, B0=B0, rp_h=host(rp),
                col_h=host(col), B0_h=host(B0), prm=prm)


def _solid(ctx, s, precision, law, v=None, H=None):
    c = s["c"]
    return api.TLSolid(ctx, s["d"], cuda(s["r0"]), cuda(s["vol"]), s["B0"], s["fixed"], s["rp"], s["col"],
                       s["v"] if v is None else v, c["dt"], c["rho0"], c["lam"], c["G"], law=law,
                       precision=precision, H=H)


def _F_from_H(H):
    n = H.shape[1]
    d = int(round(np.sqrt(H.shape[0])))
    return np.eye(d)[None] + H.T.reshape(n, d, d)


@pytest.mark.parametrize("law", [OT.SVK, OT.NEO_HOOKEAN])
def test_rates_parity(ctx, law):
    s = _setup(ctx, law=law)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(5)
    H = 0.01 * rng.normal(size=(9, n))
    v = s["v"] + 0.1 * rng.normal(size=s["v"].shape)
    F = _F_from_H(H)
    M = OT.stress_matrix(F, s["B0_h"], s["prm"])
    a_o = OT.momentum_rate(s["r0"], s["vol"], M, s["rp_h"], s["col_h"], s["prm"].dom, s["prm"].rho0)
    Fd_o = OT.deformation_rate(s["r0"], s["vol"], v, s["B0_h"], s["rp_h"], s["col_h"], s["prm"].dom)
    Fd_o = Fd_o.reshape(n, 9).T
    for prec, tol, err in ((api.SPH_FP64, 1e-12, rel_max), (api.SPH_FP32_KAHAN, 1e-5, rel_l2)):
        sol = _solid(ctx, s, prec, law, v=v, H=H)
        a, Fd = sol.rates()
        assert err(host(a), a_o) < tol, (prec, err(host(a), a_o))
        assert err(host(Fd), Fd_o) < tol, (prec, err(host(Fd), Fd_o))


@pytest.mark.parametrize("kappa", [1.6, 2.0])
def test_steps_parity(ctx, kappa):
    s = _setup(ctx, kappa=kappa)
    n = s["r0"].shape[1]
    F0 = np.tile(np.eye(3), (n, 1, 1))
    x_o, v_o, F_o = OT.run(s["r0"], s["vol"], s["B0_h"], s["fixed"], s["r0"].copy(), s["v"], F0, s["rp_h"],
                           s["col_h"], s["prm"], 20)
    H_o = (F_o - np.eye(3)[None]).reshape(n, 9).T
    for prec, tol, err in ((api.SPH_FP64, 1e-12, rel_max), (api.SPH_FP32_KAHAN, 1e-5, rel_l2)):
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN)
        sol.step(20)
        x, v, H = sol.fields()
        assert err(host(v), v_o) < tol, (prec, err(host(v), v_o))
        assert err(host(H), H_o) < tol, (prec, err(host(H), H_o))
        assert err(host(x) - s["r0"], x_o - s["r0"]) < tol
        assert np.all(host(v)[:, s["fixed"] == 1] == 0.0)


def test_linear_field_and_momentum_invariants(ctx):
    s = _setup(ctx)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(2)
    L = 0.3 * rng.normal(size=(3, 3))
    v = L @ s["r0"] + 0.2
    sol = _solid(ctx, s, api.SPH_FP64, OT.NEO_HOOKEAN, v=v, H=0.01 * rng.normal(size=(9, n)))
    a, Fd = sol.rates()
    a, Fd = host(a), host(Fd).T.reshape(n, 3, 3)
    assert np.max(np.abs(Fd - L[None])) < 1e-9 * np.max(np.abs(L))
    tot = np.sum(s["vol"] * a, axis=1)
    assert np.max(np.abs(tot)) < 1e-12 * np.sum(s["vol"] * np.abs(a))


def test_full_size_plate_sampled(ctx):
    # the 816k-particle plate (dp = 1 mm) as benchmarked: float32 rates on sampled rows
    s = _setup(ctx, dp=0.001)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(7)
    H = 0.01 * rng.normal(size=(9, n))
    sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN, H=H)
    a, Fd = sol.rates()
    a, Fd = host(a), host(Fd)
    rows = rng.choice(n, 64, replace=False)
    nb = np.unique(np.concatenate([rows, s["col_h"][np.concatenate([np.arange(s["rp_h"][i], s["rp_h"][i + 1])
                                                                    for i in rows])]]))
    Fm = np.tile(np.eye(3), (n, 1, 1))
    Fm[nb] = _F_from_H(H[:, nb])
    M = np.zeros((n, 3, 3))
    M[nb] = OT.stress_matrix(Fm[nb], s["B0_h"][:, nb], s["prm"])
    rp_s, col_s = sample_rows(s["rp_h"], s["col_h"], rows)
    a_o = OT.momentum_rate(s["r0"], s["vol"], M, rp_s, col_s, s["prm"].dom, s["prm"].rho0)
    Fd_o = OT.deformation_rate(s["r0"], s["vol"], s["v"], s["B0_h"], rp_s, col_s, s["prm"].dom).reshape(n, 9).T
    assert rel_l2(a[:, rows], a_o[:, rows]) < 1e-5
    assert rel_l2(Fd[:, rows], Fd_o[:, rows]) < 1e-5
