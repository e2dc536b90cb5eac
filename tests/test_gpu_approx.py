"""GPU parity of the error-analysis pieces (Sec. 2.3.3) against the float64 oracle: the
2D relaxation of the circle with the Laguerre-Gauss or the standard Wendland kernel, and
the kernel summation and weak-form gradient with and without the correction matrix."""
import numpy as np
import pytest

from helpers import cuda, host, odom, rel_fp64, rel_max, sorted_by_cells
from oracle import approx as OA
from oracle import kernels as OKer
from oracle import kgc as OK
from oracle import neighbors as ON
from oracle import relax as OR
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu

KINDS = {api.SPH_LAGUERRE_GAUSS: OKer.LAGUERRE_GAUSS, api.SPH_WENDLAND_C2: OKer.WENDLAND}


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _circle(n=20, jitter=0.25, seed=2):
    b = inputs.circle_body(2.0 / n, jitter=jitter, seed=seed)
    pos, _ = sorted_by_cells(b["pos"], b["domain"])
    return b, pos


@pytest.mark.parametrize("kernel", [api.SPH_LAGUERRE_GAUSS, api.SPH_WENDLAND_C2])
def test_2d_relaxation_parity(ctx, kernel):
    b, pos = _circle()
    dom = odom(b["domain"])
    kind = KINDS[kernel]
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP64, kernel=kernel)
    rp, col = ON.neighbors_cells(pos, dom)
    a_o = OR.acceleration(pos, b["vol"], rp, col, dom, b["spheres"], kind=kind)
    a = api.relax_accel(ctx, prm, cuda(pos), cuda(b["vol"]))
    assert rel_fp64(host(a), a_o) < 1e-12
    x_o = OR.run(pos, b["vol"], dom, b["spheres"], b["dp"], 4, kind=kind)
    x = cuda(pos).clone()
    api.relax_step(ctx, prm, x, cuda(b["vol"]), 4)
    assert np.max(np.abs(host(x) - x_o)) < 1e-12 * b["dp"]
    # the residual (Laguerre-Gauss and truncated Wendland sums over phi < -2h) in 2D
    r_o = OR.residual(x_o, b["vol"], dom, b["spheres"])
    r = api.relax_residual(ctx, prm, x, cuda(b["vol"]))
    assert r[2] == r_o[2] and abs(r[0] - r_o[0]) <= 1e-11 * r_o[0] and abs(r[1] - r_o[1]) <= 1e-11 * r_o[1]


def test_float32_relaxation_is_3d_laguerre_gauss_only(ctx):
    b, pos = _circle()
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP32_KAHAN)
    with pytest.raises(api.L.SphError):
        api.relax_step(ctx, prm, cuda(pos), cuda(b["vol"]), 1)


@pytest.mark.parametrize("kappa", [2.0, 1.6])
@pytest.mark.parametrize("dist", ["lattice", "jittered", "periodic"])
def test_field_approximations_parity(ctx, kappa, dist):
    if dist == "periodic":
        n = 24
        dp = 1.0 / n
        pos = inputs.lattice((n, n), dp)
        d = inputs.domain(2, 1.3 * dp, kappa, [0.0, 0.0], [1.0, 1.0], (True, True))
        vol = np.full(pos.shape[1], dp * dp)
    else:
        b, pos = _circle(jitter=0.0 if dist == "lattice" else 0.3, seed=5)
        d = dict(b["domain"])
        d["kappa"] = kappa
        vol = b["vol"]
    dom = odom(d)
    rp, col = ON.neighbors_cells(pos, dom)
    rp_d, col_d = api.build_neighbors(ctx, d, cuda(pos))
    assert np.array_equal(host(rp_d), rp) and np.array_equal(host(col_d), col)
    B_o, fb = OK.kgc(pos, vol, rp, col, dom, OKer.WENDLAND)
    B, _, _ = api.kgc(ctx, d, cuda(pos), cuda(vol), rp_d, col_d)
    f = np.exp(-pos[0] ** 2 / 0.1) + 0.3 * pos[1]
    for with_b in (False, True):
        s, g = api.field_approx(ctx, d, cuda(pos), cuda(vol), rp_d, col_d, cuda(f), B=B if with_b else None)
        s_o = OA.kernel_sum(pos, vol, f, rp, col, dom)
        g_o = OA.weak_gradient(pos, vol, f, rp, col, dom, B=B_o if with_b else None)
        assert rel_fp64(host(s), s_o) < 1e-12
        assert rel_fp64(host(g), g_o) < 1e-12, (with_b, rel_fp64(host(g), g_o))
