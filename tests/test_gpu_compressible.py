"""GPU parity of the compressible Riemann SPH path (Sec. 3.1, HLLC with the dissipation
limiter) against the float64 oracle.

Each side builds its own neighbour list and correction matrices from the same positions,
so the whole chain (list, Eq. 27, Eq. 18 with Eqs. 20-24) is compared.  float64 fields must
agree within 1e-12 (normwise relative) after one evaluation, 1e-10 after tens of steps;
the float32 form's rates within 1e-5 relative L2 (Eq. 10 form), and so must the change of
its float64 state over a run."""
import numpy as np
import pytest

from helpers import cuda, host, odom, oracle_rows, rel_fp64, rel_l2, rel_max, sample_rows, sorted_by_cells
from oracle import compressible as OC
from oracle import kgc as OK
from oracle import neighbors as ON
from paper_2405_05155_gb300 import _lib as L
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _state(n, dim, seed, collide=1.0):
    """Random gas states: rho in [0.5, 2], v with components ~ N(0, 0.5) (|v| of the order
    of c, so colliding pairs reach the limiter's cap and the crossing-wave branch), p in
    [0.3, 3]."""
    rng = np.random.default_rng(seed)
    rho = rng.uniform(0.5, 2.0, n)
    v = collide * 0.5 * rng.normal(size=(dim, n))
    p = rng.uniform(0.3, 3.0, n)
    return rho, rho * v, p / 0.4 + 0.5 * rho * np.sum(v * v, axis=0)


def _periodic(dim, m, kappa, jitter=0.3, seed=0):
    dp = 1.0 / m
    pos = inputs.lattice((m,) * dim, dp)
    rng = np.random.default_rng(seed)
    pos = np.mod(pos + rng.uniform(-jitter, jitter, pos.shape) * dp, 1.0)
    d = inputs.domain(dim, inputs.H_FLUID * dp, kappa, (0.0,) * dim, (1.0,) * dim, (True,) * dim)
    pos, _ = sorted_by_cells(pos, d)
    return pos, np.full(pos.shape[1], dp ** dim), d


def _both(ctx, pos, vol, d):
    """(device list + correction, oracle list + correction) built independently."""
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    B, _, _ = api.kgc(ctx, d, cuda(pos), cuda(vol), rp, col)
    od = odom(d)
    orp, ocol = ON.neighbors_cells(pos, od)
    oB, _ = OK.kgc(pos, vol, orp, ocol, od)
    return (rp, col, B), (orp, ocol, oB, od)


def _sim(ctx, d, pos, vol, dev, rho, mom, E, dt, eta=1.0, precision=api.SPH_FP64):
    rp, col, B = dev
    return api.Compressible(ctx, d, cuda(pos), cuda(vol), B, rp, col, rho, mom, E, dt, eta=eta, precision=precision)


# (precision, tolerance, measure) of the rates
FORMS = ((api.SPH_FP64, 1e-12, rel_fp64), (api.SPH_FP32_KAHAN, 1e-5, rel_l2))


@pytest.mark.parametrize("dim,m", [(2, 24), (3, 9)])
@pytest.mark.parametrize("kappa", [1.6, 2.0])
@pytest.mark.parametrize("form", FORMS, ids=["fp64", "fp32"])
def test_rates_parity(ctx, dim, m, kappa, form):
    prec, tol, err = form
    pos, vol, d = _periodic(dim, m, kappa, seed=dim)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], dim, seed=10 + dim)
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4, precision=prec)
    got = [host(t) for t in sim.rates()]
    want = OC.compressible_rates(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, 1e-4))
    for g, w in zip(got, want):
        assert err(g, w) < tol, err(g, w)


@pytest.mark.parametrize("eta", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("form", FORMS, ids=["fp64", "fp32"])
def test_limiter_strengths(ctx, eta, form):
    # eta = 0 removes the dissipation (beta = 0: u* and p* are the impedance-weighted and
    # plain means), eta = 1 is the paper's setting
    prec, tol, err = form
    pos, vol, d = _periodic(2, 20, 1.6, seed=5)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], 2, seed=6, collide=2.0)
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4, eta=eta, precision=prec)
    got = [host(t) for t in sim.rates()]
    want = OC.compressible_rates(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, 1e-4, eta=eta))
    for g, w in zip(got, want):
        assert err(g, w) < tol, err(g, w)


@pytest.mark.parametrize("dim,m", [(2, 24), (3, 9)])
def test_fp32_lane_shapes(ctx, dim, m):
    # 1 to 8 lanes per row: the same pairs, partial sums combined by shuffles; every
    # shape within the float32 tolerance of the oracle, and 20 steps of each agree
    pos, vol, d = _periodic(dim, m, 2.0, seed=11)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], dim, seed=12)
    want = OC.compressible_rates(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, 1e-4))
    ends = []
    try:
        for lanes in (1, 2, 4, 8):
            ctx.set_lanes(api.SPH_PASS_COMPRESSIBLE, lanes)
            sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4, precision=api.SPH_FP32_KAHAN)
            for g, w in zip((host(t) for t in sim.rates()), want):
                assert rel_l2(g, w) < 1e-5, (lanes, rel_l2(g, w))
            sim.step(20)
            ends.append(host(sim.E) - E)
    finally:
        ctx.set_lanes(api.SPH_PASS_COMPRESSIBLE, 1)
    for x in ends[1:]:
        assert rel_l2(x, ends[0]) < 1e-5


def test_fp32_steps_and_conservation(ctx):
    # 20 float32 steps: the change of the float64 state against the oracle's, and the
    # totals (sums of float32 rates: conserved to float32 rounding of the fluxes)
    pos, vol, d = _periodic(3, 10, 1.6, seed=9)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], 3, seed=2, collide=0.5)
    dt = 2e-4
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, dt, precision=api.SPH_FP32_KAHAN)
    sim.step(20)
    got = (host(sim.rho), host(sim.mom), host(sim.E))
    want = OC.run(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, dt), 20)
    for g, w, x0 in zip(got, want, (rho, mom, E)):
        assert rel_l2(g - x0, w - x0) < 1e-5, rel_l2(g - x0, w - x0)
    for g, w, x0 in ((got[0], want[0], rho), (got[2], want[2], E)):
        assert abs(np.sum(vol * (g - x0))) < 1e-6 * np.sum(vol * np.abs(w - x0))


def test_long_rows_rates_parity(ctx):
    # random points in a periodic unit cube, about 180 neighbours each (plan width above 128)
    n = 1500
    rng = np.random.default_rng(31)
    pos = rng.uniform(0.0, 1.0, size=(3, n))
    d = inputs.domain(3, 0.19, 1.6, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (True, True, True))
    pos, _ = sorted_by_cells(pos, d)
    vol = np.full(n, 1.0 / n)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    assert np.max(np.diff(orp)) > 128
    rho, mom, E = _state(n, 3, seed=32)
    want = OC.compressible_rates(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, 1e-4))
    for prec, tol, err in FORMS:
        sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4, precision=prec)
        for g, w in zip((host(t) for t in sim.rates()), want):
            assert err(g, w) < tol, (prec, err(g, w))


def test_plan_arguments(ctx):
    pos, vol, d = _periodic(2, 8, 1.6)
    dev, _ = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], 2, seed=1)
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4, precision=api.SPH_FP32_KAHAN)
    assert sim.st.plan_width == int(np.max(np.diff(host(dev[0]))))
    before = host(sim.E).copy()
    good = sim.st.plan_bytes
    sim.st.plan_bytes = good - 16                    # too small for the width
    with pytest.raises(L.SphError):
        sim.step(1)
    sim.st.plan_bytes = good
    sim.st.plan_width = 0                            # no plan built
    with pytest.raises(L.SphError):
        sim.step(1)
    assert np.array_equal(host(sim.E), before)


def test_steps_parity_and_conservation(ctx):
    pos, vol, d = _periodic(2, 20, 1.6, seed=7)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], 2, seed=8, collide=0.5)
    dt = 2e-4
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, dt)
    sim.step(20)
    r1, m1, E1 = host(sim.rho), host(sim.mom), host(sim.E)
    wr, wm, wE = OC.run(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, dt), 20)
    assert rel_max(r1, wr) < 1e-10 and rel_max(m1, wm) < 1e-10 and rel_max(E1, wE) < 1e-10
    # the pairwise-antisymmetric fluxes conserve mass, momentum and energy on the device too
    for a, b in ((r1, rho), (E1, E)):
        assert abs(np.sum(vol * a) - np.sum(vol * b)) < 1e-13 * np.sum(vol * np.abs(b))
    assert np.max(np.abs(np.sum(vol * m1, axis=1) - np.sum(vol * mom, axis=1))) < 1e-13


def test_uniform_rest_is_a_fixed_point(ctx):
    pos, vol, d = _periodic(3, 8, 2.0, jitter=0.0)
    dev, _ = _both(ctx, pos, vol, d)
    n = pos.shape[1]
    sim = _sim(ctx, d, pos, vol, dev, np.ones(n), np.zeros((3, n)), np.full(n, 2.5), 1e-3)
    dr, dm, dE = (host(t) for t in sim.rates())
    assert np.max(np.abs(dr)) < 1e-12 and np.max(np.abs(dm)) < 1e-11 and np.max(np.abs(dE)) < 1e-11


def _sod(ctx, nx, ny, kappa):
    c = inputs.sod_strip(nx=nx, ny=ny, kappa=kappa)
    d = c["domain"]
    pos, order = sorted_by_cells(c["pos"], d)
    return c, d, pos, c["vol"][order], c["rho"][order], c["mom"][:, order], c["E"][order]


@pytest.mark.parametrize("kappa", [1.6, 2.0])
def test_sod_strip_parity(ctx, kappa):
    # the whole run to t = 0.1 (192 steps): float64 within 1e-10, float32 within 1e-5 of
    # the state's change
    c, d, pos, vol, rho, mom, E = _sod(ctx, 200, 6, kappa)
    dev, (orp, ocol, oB, od) = _both(ctx, pos, vol, d)
    steps = int(round(0.1 / c["dt"]))
    want = OC.run(pos, vol, rho, mom, E, oB, orp, ocol, OC.CompressibleParams(od, c["dt"]), steps)
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, c["dt"])
    sim.step(steps)
    got = (host(sim.rho), host(sim.mom), host(sim.E))
    for g, w in zip(got, want):
        assert rel_max(g, w) < 1e-10
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, c["dt"], precision=api.SPH_FP32_KAHAN)
    sim.step(steps)
    got = (host(sim.rho), host(sim.mom), host(sim.E))
    for g, w, x0 in zip(got, want, (rho, mom, E)):
        assert rel_l2(g - x0, w - x0) < 1e-5, rel_l2(g - x0, w - x0)


def test_sod_strip_converges_to_the_exact_solution(ctx):
    # a property at any size: the L1 density error against the exact Riemann solution
    # falls as dp falls (first order at the discontinuities)
    errs = []
    for nx in (200, 800):
        c, d, pos, vol, rho, mom, E = _sod(ctx, nx, 6, 1.6)
        dev, _ = _both(ctx, pos, vol, d)
        steps = int(round(0.1 / c["dt"]))
        sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, c["dt"])
        sim.step(steps)
        x = pos[0]
        sel = (x > 0.3) & (x < 0.8)
        ex, _, _, _, _ = OC.exact_riemann(1.0, 0.0, 1.0, 0.125, 0.0, 0.1, (x[sel] - 0.5) / (steps * c["dt"]))
        r = host(sim.rho)
        assert np.all(np.isfinite(r)) and np.all(r > 0)
        errs.append(np.mean(np.abs(r[sel] - ex)))
    assert errs[0] < 0.02 and errs[1] < 0.6 * errs[0], errs


def test_full_size_sampled_rows(ctx):
    # the bench workload's geometry (a 4096 x 64 Sod strip, kappa = 1.6, 262,144 particles)
    # at a random gas state, in the launch shape the step uses; the oracle evaluates 96
    # sampled rows (its list and correction built for those rows and their neighbours)
    c, d, pos, vol, _, _, _ = _sod(ctx, 4096, 64, 1.6)
    n = pos.shape[1]
    rho, mom, E = _state(n, 2, seed=4)
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    B, _, _ = api.kgc(ctx, d, cuda(pos), cuda(vol), rp, col)
    forms = []
    for prec in (api.SPH_FP64, api.SPH_FP32_KAHAN):
        sim = _sim(ctx, d, pos, vol, (rp, col, B), rho, mom, E, c["dt"], precision=prec)
        forms.append([host(t) for t in sim.rates()])
        del sim
    rows = np.unique(np.concatenate([np.random.default_rng(0).choice(n, 64, replace=False),
                                     np.argsort(np.abs(pos[0] - 0.5))[:32]]))
    od = odom(d)
    orp, ocol, oB, _ = oracle_rows(pos, vol, od, rows, 1)
    srp, scol = sample_rows(orp, ocol, rows)
    want = OC.compressible_rates(pos, vol, rho, mom, E, oB, srp, scol, OC.CompressibleParams(od, c["dt"]))
    for (prec, tol, err), got in zip(FORMS, forms):
        for g, w in zip(got, want):
            assert err(g[..., rows], w[..., rows]) < tol, (prec, err(g[..., rows], w[..., rows]))


def test_arguments_and_degenerate_sizes(ctx):
    pos, vol, d = _periodic(2, 8, 1.6)
    dev, _ = _both(ctx, pos, vol, d)
    rho, mom, E = _state(pos.shape[1], 2, seed=1)
    sim = _sim(ctx, d, pos, vol, dev, rho, mom, E, 1e-4)
    before = host(sim.E).copy()
    sim.step(0)                                   # no step: state untouched
    assert np.array_equal(host(sim.E), before)
    for field, bad in (("gamma", 1.0), ("dt", -1.0), ("eta", -0.5), ("precision", 99)):
        old = getattr(sim.prm, field)
        setattr(sim.prm, field, bad)
        with pytest.raises(L.SphError):
            sim.step(1)
        setattr(sim.prm, field, old)
    with pytest.raises(L.SphError):
        sim.step(-1)
    assert np.array_equal(host(sim.E), before)
    # an empty set is a no-op
    empty = np.zeros((2, 0))
    z = api.Compressible(ctx, d, cuda(empty), cuda(np.zeros(0)), cuda(np.zeros((3, 0))), dev[0][:1] * 0, dev[1][:0],
                         np.zeros(0), empty, np.zeros(0), 1e-4)
    z.step(3)
    assert all(t.numel() == 0 for t in z.rates())
