"""GPU parity of the Laguerre-Gauss relaxation (a10, a11) against the float64 oracle."""
import numpy as np
import pytest

from helpers import cuda, host, odom, rel_l2, rel_max, sorted_by_cells
from oracle import neighbors as ON
from oracle import relax as OR
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _body(seed=3, dp=1.0 / 24.0):
    b = inputs.sphere_body(seed, dp)
    pos, _ = sorted_by_cells(b["pos"], b["domain"])
    return b, pos


def test_acceleration_parity(ctx):
    b, pos = _body()
    dom = odom(b["domain"])
    rp, col = ON.neighbors_cells(pos, dom)
    a_o = OR.acceleration(pos, b["vol"], rp, col, dom, b["spheres"])
    for prec, tol, err in ((api.SPH_FP64, 1e-12, rel_max), (api.SPH_FP32_KAHAN, 1e-4, rel_l2)):
        prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=prec)
        a = api.relax_accel(ctx, prm, cuda(pos), cuda(b["vol"]))
        assert err(host(a), a_o) < tol, (prec, err(host(a), a_o))


def test_steps_parity_float64(ctx):
    b, pos = _body()
    dom = odom(b["domain"])
    x_o = OR.run(pos, b["vol"], dom, b["spheres"], b["dp"], 3)
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP64)
    x = cuda(pos).clone()
    api.relax_step(ctx, prm, x, cuda(b["vol"]), 3)
    assert np.max(np.abs(host(x) - x_o)) < 1e-12 * b["dp"]


def test_steps_float32_from_identical_state(ctx):
    # float32 pair sums: each step compared from the same float64 state
    b, pos = _body(seed=4)
    dom = odom(b["domain"])
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP32_KAHAN)
    cur = pos
    for _ in range(3):
        x_o = OR.step(cur, b["vol"], dom, b["spheres"], b["dp"])
        x = cuda(cur).clone()
        api.relax_step(ctx, prm, x, cuda(b["vol"]), 1)
        x = host(x)
        # displacements agree to float32 accuracy (relative to the step size h/32)
        assert np.max(np.abs(x - x_o)) < 1e-3 * b["h"] / 32.0 + 1e-12
        cur = x_o


def test_residual_parity_and_decrease(ctx):
    b, pos = _body(seed=6, dp=1.0 / 28.0)
    dom = odom(b["domain"])
    prm = api.relax_params(b["domain"], b["spheres"], b["dp"], precision=api.SPH_FP32_KAHAN)
    r_o = OR.residual(pos, b["vol"], dom, b["spheres"])
    r = api.relax_residual(ctx, prm, cuda(pos), cuda(b["vol"]))
    assert r[2] == r_o[2]
    assert abs(r[0] - r_o[0]) < 1e-12 * r_o[0] and abs(r[1] - r_o[1]) < 1e-12 * r_o[1]
    x = cuda(pos).clone()
    api.relax_step(ctx, prm, x, cuda(b["vol"]), 40)
    r1 = api.relax_residual(ctx, prm, x, cuda(b["vol"]))
    assert r1[0] < 0.4 * r[0]
    phi, _ = OR.sdf_spheres(host(x), b["spheres"])
    # float32 signed distance: the projection lands on -dp/2 to ~1e-7 of the sphere radius
    assert np.all(phi <= -0.5 * b["dp"] + 1e-5 * b["dp"])


def test_capacity_regrowth(ctx):
    # a body denser than the default list capacity forces a mid-run regrow; the
    # result must equal an uninterrupted float64 run
    b, pos = _body(seed=8, dp=1.0 / 20.0)
    d = dict(b["domain"])
    d["h"] = 4.0 * b["dp"]          # ~1100 neighbours per particle at cut-off 2h, above 128
    dom = odom(d)
    prm = api.relax_params(d, b["spheres"], b["dp"], precision=api.SPH_FP64)
    x = cuda(pos).clone()
    api.relax_step(ctx, prm, x, cuda(b["vol"]), 2)
    x_o = OR.run(pos, b["vol"], dom, b["spheres"], b["dp"], 2)
    assert np.max(np.abs(host(x) - x_o)) < 1e-12
