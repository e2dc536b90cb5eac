"""GPU parity of the Eulerian WCSPH path (a5, a6) against the float64 oracle.

float64 fields must agree within 1e-12 (normwise relative), float32 fields within
1e-5 relative L2 (Eq. 10 form)."""
import math

import numpy as np
import pytest
import torch

from helpers import cuda, host, odom, oracle_rows, OracleLists, rel_elem, rel_fp64, rel_l2, rel_max, sample_rows, sorted_by_cells
from oracle import eulerian as OE
from oracle import kgc as OK
from oracle import neighbors as ON
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _setup(ctx, case, jitter=0.0, seed=0, sort=True):
    d = case["domain"]
    pos = case["pos"]
    if jitter:
        rng = np.random.default_rng(seed)
        pos = np.mod(pos + rng.uniform(-jitter, jitter, pos.shape) * case["dp"], d["len"][0])
    order = np.arange(pos.shape[1])
    if sort:
        pos, order = sorted_by_cells(pos, d)
    v = case["v"][:, order]
    drho = (case["p"] / case["c0"] ** 2)[order]
    vol = case["vol"][order]
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    B, fb, _ = api.kgc(ctx, d, cuda(pos), cuda(vol), rp, col)
    prm = OE.EulerianParams(odom(d), case["dt"], case["rho0"], case["c0"], case["mu"])
    return OracleLists("pos", "B_h", pos=pos, vol=vol, v=v, drho=drho, rp=rp, col=col, B=B, prm=prm, d=d)


def _sim(ctx, s, case, precision, integrator=api.SPH_TWO_PASS, drho=None, v=None, tiles=True):
    return api.Eulerian(ctx, s["d"], cuda(s["pos"]), cuda(s["vol"]), s["B"], s["rp"], s["col"],
                        s["drho"] if drho is None else drho, s["v"] if v is None else v, case["dt"],
                        case["rho0"], case["c0"], case["mu"], precision=precision, integrator=integrator,
                        tiles=tiles)


# float64; float32 on the tile plan (precomputed pair geometry); float32 evaluating
# the geometry per pair from the records
VARIANTS = ((api.SPH_FP64, True, 1e-12, rel_fp64), (api.SPH_FP32_KAHAN, True, 1e-5, rel_l2),
            (api.SPH_FP32_KAHAN, False, 1e-5, rel_l2))


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kappa", [1.6, 2.0])
def test_rates_parity(ctx, dim, kappa):
    case = inputs.tgv2d(nx=32, kappa=kappa) if dim == 2 else inputs.tgv3d(n=12, kappa=kappa)
    s = _setup(ctx, case, jitter=0.2, seed=dim)
    rng = np.random.default_rng(9)
    drho = s["drho"] + 1e-3 * rng.normal(size=s["drho"].shape)
    v = s["v"] + 0.1 * rng.normal(size=s["v"].shape)
    ro, mo = OE.eulerian_rates(s["pos"], s["vol"], drho, v, s["B_h"], s["rp_h"], s["col_h"], s["prm"])
    for prec, tiles, tol, err in VARIANTS:
        sim = _sim(ctx, s, case, prec, drho=drho, v=v, tiles=tiles)
        r, m = sim.rates()
        assert err(host(r), ro) < tol, (prec, err(host(r), ro))
        assert err(host(m), mo) < tol, (prec, err(host(m), mo))


def test_long_rows_rates_parity(ctx):
    # random points in a periodic unit cube with about 180 neighbours each (rows above the
    # 128 pairs the plan's offset ordering handles): every form against the oracle
    n = 1500
    rng = np.random.default_rng(21)
    pos = rng.uniform(0.0, 1.0, size=(3, n))
    h = 0.19
    case = {"domain": inputs.domain(3, h, 1.6, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (True, True, True)),
            "pos": pos, "dp": 1.0 / n ** (1.0 / 3.0), "v": 0.1 * rng.normal(size=(3, n)),
            "p": 0.01 * rng.normal(size=n), "c0": 1.0, "vol": np.full(n, 1.0 / n), "dt": 1e-3, "rho0": 1.0,
            "mu": 0.01}
    s = _setup(ctx, case)
    assert np.max(np.diff(host(s["rp"]))) > 128
    ro, mo = OE.eulerian_rates(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"])
    for prec, tiles, tol, err in VARIANTS:
        sim = _sim(ctx, s, case, prec, tiles=tiles)
        r, m = sim.rates()
        assert err(host(r), ro) < tol, (prec, tiles, err(host(r), ro))
        assert err(host(m), mo) < tol, (prec, tiles, err(host(m), mo))


def test_plain_method_tgv2d_200_steps(ctx):
    # 2D Taylor-Green vortex, 50x50, h = 1.3 dp, kappa = 1.6, Re = 100, 200 steps in float64
    case = inputs.tgv2d(nx=50, kappa=1.6)
    s = _setup(ctx, case)
    d_o, v_o = OE.run(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"], 200)
    sim = _sim(ctx, s, case, api.SPH_FP64)
    sim.step(200)
    dr, v = sim.fields()
    assert rel_max(host(dr), d_o) < 1e-12
    assert rel_max(host(v), v_o) < 1e-12
    # closed-form decay exp(-8 pi^2 t / Re) of the velocity amplitude
    t = 200 * case["dt"]
    amp = np.sqrt(np.mean(host(v) ** 2)) / np.sqrt(np.mean(s["v"] ** 2))
    assert abs(amp / math.exp(-case["decay_rate"] * t) - 1.0) < 0.03
    # float32 + Kahan against the float64 oracle, same 200 steps
    for tiles in (True, False):
        sim32 = _sim(ctx, s, case, api.SPH_FP32_KAHAN, tiles=tiles)
        sim32.step(200)
        dr32, v32 = sim32.fields()
        assert rel_l2(host(v32), v_o) < 1e-5, tiles
        assert rel_l2(host(dr32), d_o) < 1e-5, (tiles, rel_l2(host(dr32), d_o))


@pytest.mark.parametrize("integrator", [api.SPH_TWO_PASS, api.SPH_FUSED])
def test_steps_3d_both_integrators(ctx, integrator):
    case = inputs.tgv3d(n=16, kappa=1.6)
    s = _setup(ctx, case)
    run = OE.run(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"], 7,
                 fused=integrator == api.SPH_FUSED)
    for prec, tiles, tol, err in VARIANTS:
        sim = _sim(ctx, s, case, prec, integrator, tiles=tiles)
        sim.step(7)
        dr, v = sim.fields()
        assert err(host(dr), run[0]) < tol and err(host(v), run[1]) < tol


def test_tgv3d_32_cubed_twenty_steps(ctx):
    # the 3D Taylor-Green case at 32^3 (Re = 1600, 1.6h) over 20 two-pass steps: float64
    # within 1e-12 normwise and element by element (each element against its own size down
    # to 1e-3 of the field's), float32 + Kahan on the tile plan within 1e-5 relative L2
    case = inputs.tgv3d(n=32, kappa=1.6)
    s = _setup(ctx, case)
    d_o, v_o = OE.run(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"], 20)
    sim = _sim(ctx, s, case, api.SPH_FP64)
    sim.step(20)
    dr, v = sim.fields()
    dr, v = host(dr), host(v)
    assert rel_max(dr, d_o) < 1e-12 and rel_max(v, v_o) < 1e-12
    assert rel_elem(dr, d_o) < 1e-10 and rel_elem(v, v_o) < 1e-10, (rel_elem(dr, d_o), rel_elem(v, v_o))
    sim = _sim(ctx, s, case, api.SPH_FP32_KAHAN)
    sim.step(20)
    dr, v = sim.fields()
    assert rel_l2(host(v), v_o) < 1e-5
    # the change of the density offset over the run (the offset itself is small and smooth)
    assert rel_l2(host(dr) - s["drho"], d_o - s["drho"]) < 1e-4


@pytest.mark.parametrize("lanes", [1, 2, 4, 8])
def test_launch_shapes_agree(ctx, lanes):
    # every launch shape (lanes per particle) meets the float32 field tolerance; the input is
    # not cell-sorted, which the neighbour builder must still turn into ascending rows
    case = inputs.tgv2d(nx=40, kappa=1.6)
    s = _setup(ctx, case, sort=False)
    d_o, v_o = OE.run(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"], 5)
    ctx.set_lanes(api.SPH_PASS_EULERIAN, lanes)
    try:
        # the lanes apply to the per-pair form; the planned form (one thread per row) on the
        # same unsorted input, whose tiles are not compact, must meet the tolerance too
        for tiles in (False, True):
            sim = _sim(ctx, s, case, api.SPH_FP32_KAHAN, tiles=tiles)
            sim.step(5)
            dr, v = sim.fields()
            assert rel_l2(host(dr), d_o) < 1e-5 and rel_l2(host(v), v_o) < 1e-5, tiles
    finally:
        ctx.set_lanes(api.SPH_PASS_EULERIAN, 4)


def test_plan_geometry_and_forms(ctx):
    # the plan's pair entries against float64 numpy on the same lists (G, viscous factor,
    # normal, slot), and the planned pass with its neighbours staged or read from global
    # memory (stage capacity 16), its entries through the thread ring or the TMA chunk
    # ring: identical arithmetic, identical results
    case = inputs.tgv3d(n=12, kappa=1.6)
    s = _setup(ctx, case, jitter=0.2, seed=5)
    n = s["pos"].shape[1]
    rp, col = host(s["rp"]), host(s["col"])           # the lists the plan was built from
    lens = np.diff(rp)
    sim = _sim(ctx, s, case, api.SPH_FP32_KAHAN)
    raw = host(sim.plan)
    nt = (n + 127) // 128
    a16 = lambda x: (x + 15) // 16 * 16
    o = 64 + 2 * a16(4 * nt)
    tile_so = raw[o:o + 8 * (nt + 1)].view(np.int64)
    o += a16(8 * (nt + 1)) + a16(4 * col.size) + a16(2 * col.size)
    o = (o + 31) // 32 * 32
    geo = raw[o:o + 32 * int(tile_so[-1])].view(np.float32).reshape(-1, 8)
    prm = s["prm"]
    dom = prm.dom
    h = dom.h
    from oracle import kernels as OKer
    B = s["B_h"]
    for i in range(0, n, 37):
        t, r = i // 128, i % 128
        ent = geo[tile_so[t] + np.arange(lens[i]) * 128 + r]
        j = col[rp[i]:rp[i + 1]]
        dx = ON.min_image(s["pos"][:, i:i + 1] - s["pos"][:, j], dom)
        d2 = np.sum(dx * dx, axis=0)
        rr = np.sqrt(d2)
        gs = OKer.wendland_dwdr(rr, h, 3, None) / rr
        Bi = OK.sym_to_full(B[:, i:i + 1], 3)[0]
        Bj = OK.sym_to_full(B[:, j], 3)
        g = np.einsum("kab,bk->ak", 0.5 * (Bi[None] + Bj), gs * dx)
        G = -2.0 * s["vol"][j] * g
        vis = 2.0 * prm.mu * s["vol"][j] * gs * d2 / (d2 + 0.01 * h * h)
        c = np.clip(np.rint(dx * (2.0 * (1.0 / h))), -8, 7).astype(np.int64) + 8
        order = np.lexsort((np.arange(j.size), (c[2] * 16 + c[1]) * 16 + c[0]))
        scale = np.abs(G).max()
        assert np.allclose(ent[:, :3].T, G[:, order], rtol=1e-6, atol=1e-6 * scale)
        assert np.allclose(ent[:, 3], vis[order], rtol=1e-6, atol=1e-6 * np.abs(vis).max())
        assert np.allclose(ent[:, 4:7].T, (-dx / rr)[:, order], rtol=1e-6, atol=1e-7)
    ref = None
    for ring in (api.SPH_RING_THREAD, api.SPH_RING_CHUNK):
        ctx.set_entry_ring(ring)
        for cap in (0, 16):
            ctx.set_stage_cap(cap)
            sim = _sim(ctx, s, case, api.SPH_FP32_KAHAN)
            sim.step(3)
            sim.unpack()                           # also reads the chunk ring's timeout flag
            got = sim.rec.clone()
            if ref is None:
                ref = got
            else:
                assert torch.equal(got, ref), (ring, cap)
    ctx.set_stage_cap(0)
    ctx.set_entry_ring(api.SPH_RING_AUTO)


def test_conservation_on_gpu(ctx):
    case = inputs.tgv3d(n=16, kappa=1.6)
    s = _setup(ctx, case, jitter=0.25, seed=4)
    rng = np.random.default_rng(1)
    v = rng.normal(size=s["v"].shape)
    sim = _sim(ctx, s, case, api.SPH_FP64, v=v)
    r, m = sim.rates()
    r, m = host(r), host(m)
    assert abs(np.sum(s["vol"] * r)) < 1e-12 * np.sum(s["vol"] * np.abs(r))
    assert np.max(np.abs(np.sum(s["vol"] * m, axis=1))) < 1e-12 * np.sum(s["vol"] * np.abs(m))


def _oracle_two_pass_sampled(s, rows):
    """One two-pass step of the oracle evaluated only where the sampled rows need it."""
    rp, col, B, _ = oracle_rows(s["pos"], s["vol"], s["prm"].dom, rows, 2)
    nbrs = np.concatenate([col[rp[i]:rp[i + 1]] for i in rows])
    rows1 = np.unique(np.concatenate([rows, nbrs]))
    prm = s["prm"]
    rho_n = prm.rho0 + s["drho"]
    rp1, col1 = sample_rows(rp, col, rows1)
    _, dmom = OE.eulerian_rates(s["pos"], s["vol"], s["drho"], s["v"], B, rp1, col1, prm, want_mass=False)
    mom1 = rho_n * s["v"] + prm.dt * dmom
    v_half = mom1 / rho_n
    rps, cols = sample_rows(rp, col, rows)
    drho_dt, _ = OE.eulerian_rates(s["pos"], s["vol"], s["drho"], v_half, B, rps, cols, prm, want_mom=False)
    drho1 = s["drho"] + prm.dt * drho_dt
    return drho1[rows], (mom1 / (prm.rho0 + drho1))[:, rows]


def test_full_size_3d_tgv_sampled(ctx):
    # 128^3 periodic Taylor-Green (2.1M particles): one float32 time step as benchmarked,
    # against the float64 oracle's step on 64 sampled particles
    case = inputs.tgv3d(n=128, kappa=1.6)
    s = _setup(ctx, case)
    n = s["pos"].shape[1]
    assert np.all(np.diff(host(s["rp"])) == 32)
    sim = _sim(ctx, s, case, api.SPH_FP32_KAHAN)
    sim.step(1)
    dr, v = sim.fields()
    dr, v = host(dr), host(v)
    rows = np.random.default_rng(3).choice(n, 64, replace=False)
    d_o, v_o = _oracle_two_pass_sampled(s, rows)
    assert rel_l2(dr[rows], d_o) < 1e-5
    assert rel_l2(v[:, rows], v_o) < 1e-5


def test_double_shear_layer_parity(ctx):
    # the inviscid (mu = 0) double shear layer of Sec. 5 at 32^2, 20 steps: float64 and
    # float32 on the tile plan against the oracle; momentum conserved on the periodic square
    case = inputs.double_shear_layer(nx=32, kappa=1.6)
    s = _setup(ctx, case)
    d_o, v_o = OE.run(s["pos"], s["vol"], s["drho"], s["v"], s["B_h"], s["rp_h"], s["col_h"], s["prm"], 20)
    for prec, tiles, tol, err in VARIANTS:
        sim = _sim(ctx, s, case, prec, tiles=tiles)
        sim.step(20)
        dr, v = sim.fields()
        assert err(host(v), v_o) < tol and err(host(dr), d_o) < max(tol, 1e-12), (prec, tiles)
    rho = case["rho0"] + d_o
    mom = np.sum(s["vol"] * rho * v_o, axis=1)
    mom0 = np.sum(s["vol"] * case["rho0"] * s["v"], axis=1)
    assert np.max(np.abs(mom - mom0)) < 1e-12
