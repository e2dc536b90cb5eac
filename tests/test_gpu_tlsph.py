"""GPU parity of the total-Lagrangian solid path (a7-a9) against the float64 oracle."""
import numpy as np
import pytest
import torch

from helpers import cuda, host, odom, oracle_rows, OracleLists, rel_fp64, rel_l2, rel_max, sample_rows, sorted_by_cells
from oracle import kgc as OK
from oracle import neighbors as ON
from oracle import tlsph as OT
from paper_2405_05155_gb300 import _lib
from paper_2405_05155_gb300 import api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _setup(ctx, dp=0.005, kappa=1.6, law=OT.NEO_HOOKEAN, case=None):
    c = inputs.plate(dp=dp, kappa=kappa) if case is None else case
    d = c["domain"]
    r0, order = sorted_by_cells(c["r0"], d)
    v = c["v"][:, order]
    fixed = c["fixed"][order]
    vol = c["vol"][order]
    rp, col = api.build_neighbors(ctx, d, cuda(r0))
    B0, fb, _ = api.kgc(ctx, d, cuda(r0), cuda(vol), rp, col)
    prm = OT.TLParams(odom(d), c["dt"], c["rho0"], c["lam"], c["G"], law)
    return OracleLists("r0", "B0_h", c=c, d=d, r0=r0, v=v, fixed=fixed, vol=vol, rp=rp, col=col, B0=B0, prm=prm)


@pytest.fixture(autouse=True)
def _default_pipeline(ctx):
    yield
    ctx.set_tile_pipeline(api.SPH_PIPE_GEOM)


def _solid(ctx, s, precision, law, v=None, H=None, tiles=True):
    # tiles = "geom" / "stream": the tile plan, the deformation pass evaluating the pair
    # geometry from staged records (SPH_PIPE_GEOM, the default) or streaming the
    # precomputed entries (SPH_PIPE_STREAM); the mode stays in force until the test ends
    if tiles in ("geom", "stream"):
        ctx.set_tile_pipeline(api.SPH_PIPE_GEOM if tiles == "geom" else api.SPH_PIPE_STREAM)
        tiles = True
    c = s["c"]
    return api.TLSolid(ctx, s["d"], cuda(s["r0"]), cuda(s["vol"]), s["B0"], s["fixed"], s["rp"], s["col"],
                       s["v"] if v is None else v, c["dt"], c["rho0"], c["lam"], c["G"], law=law,
                       precision=precision, H=H, tiles=tiles)


# float64; float32 on the tile plan streaming its entries, float32 gathering from global
# memory, and float32 on the plan with the deformation pass's geometry per pair
VARIANTS = ((api.SPH_FP64, True, 1e-12, rel_fp64), (api.SPH_FP32_KAHAN, "stream", 1e-5, rel_l2),
            (api.SPH_FP32_KAHAN, False, 1e-5, rel_l2), (api.SPH_FP32_KAHAN, "geom", 1e-5, rel_l2))


@pytest.mark.parametrize("periodic", [False, True])
def test_2d_strip_rates_and_steps(ctx, periodic):
    # the 2D forms (clamped strip, and a strip periodic along x for the minimum image of
    # the cell-relative positions and of the plan's pair factors)
    case = inputs.beam2d(dp=0.002, periodic_x=periodic)
    s = _setup(ctx, case=case)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(11)
    H = 0.01 * rng.normal(size=(4, n))
    v = s["v"] + 0.05 * rng.normal(size=s["v"].shape)
    F = _F_from_H(H)
    M = OT.stress_matrix(F, s["B0_h"], s["prm"])
    a_o = OT.momentum_rate(s["r0"], s["vol"], M, s["rp_h"], s["col_h"], s["prm"].dom, s["prm"].rho0)
    Fd_o = OT.deformation_rate(s["r0"], s["vol"], v, s["B0_h"], s["rp_h"], s["col_h"], s["prm"].dom)
    Fd_o = Fd_o.reshape(n, 4).T
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN, v=v, H=H, tiles=tiles)
        a, Fd = sol.rates()
        assert err(host(a), a_o) < tol, (prec, tiles, err(host(a), a_o))
        assert err(host(Fd), Fd_o) < tol, (prec, tiles, err(host(Fd), Fd_o))
    F0 = np.tile(np.eye(2), (n, 1, 1))
    x_o, v_o, F_o = OT.run(s["r0"], s["vol"], s["B0_h"], s["fixed"], s["r0"].copy(), s["v"], F0, s["rp_h"],
                           s["col_h"], s["prm"], 10)
    H_o = (F_o - np.eye(2)[None]).reshape(n, 4).T
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN, tiles=tiles)
        sol.step(10)
        x, vv, HH = sol.fields()
        assert err(host(vv), v_o) < tol, (prec, tiles, err(host(vv), v_o))
        assert err(host(HH), H_o) < tol, (prec, tiles, err(host(HH), H_o))


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
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, law, v=v, H=H, tiles=tiles)
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
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN, tiles=tiles)
        sol.step(20)
        x, v, H = sol.fields()
        assert err(host(v), v_o) < tol, (prec, err(host(v), v_o))
        assert err(host(H), H_o) < tol, (prec, err(host(H), H_o))
        assert err(host(x) - s["r0"], x_o - s["r0"]) < tol
        assert np.all(host(v)[:, s["fixed"] == 1] == 0.0)


def _match_order(slots):
    """The pair order of a tile for its staged gathers, written out from its description:
    per quarter warp (8 consecutive rows) and step, a maximum matching of the active rows
    to groups (slot mod 8) in which they have pairs left, by augmenting paths with rows
    taken by most pairs left and each row trying its fullest groups first (ties to the
    lower row, the lower group); an unmatched row takes the group picked least often in
    the step, then its fullest, then the lower group; within a group, list order."""
    orders = [np.zeros(len(sl), dtype=np.int64) for sl in slots]
    for q0 in range(0, len(slots), 8):
        rows = list(range(q0, min(q0 + 8, len(slots))))
        byg = {r: [[k for k in range(len(slots[r])) if int(slots[r][k]) % 8 == g] for g in range(8)] for r in rows}
        left = {r: len(slots[r]) for r in rows}
        for p in range(max(left.values())):
            act = sorted([r for r in rows if left[r] > 0], key=lambda r: -left[r])
            owner = [None] * 8

            def augment(r, seen):
                for g in sorted(range(8), key=lambda g: -len(byg[r][g])):
                    if not byg[r][g] or g in seen:
                        continue
                    seen.add(g)
                    if owner[g] is None or augment(owner[g], seen):
                        owner[g] = r
                        return True
                return False

            for r in act:
                augment(r, set())
            pick = {owner[g]: g for g in range(8) if owner[g] is not None}
            picks = [1 if owner[g] is not None else 0 for g in range(8)]
            for r in act:
                if r not in pick:
                    g = min((g for g in range(8) if byg[r][g]), key=lambda g: (picks[g], -len(byg[r][g]), g))
                    pick[r] = g
                    picks[g] += 1
            for r in act:
                orders[r][p] = byg[r][pick[r]].pop(0)
                left[r] -= 1
    return orders


def _read_plan(plan, n, nnz, maxrow):
    """Split a tile-plan buffer by its documented layout."""
    raw = host(plan)
    nt = (n + 127) // 128
    a16 = lambda x: (x + 15) // 16 * 16
    out = {"hdr": raw[:64].view(np.int32)}
    o = 64
    for name, size, dt in (("tile_m", 4 * nt, np.int32), ("tile_e", 4 * nt, np.int32),
                           ("tile_so", 8 * (nt + 1), np.int64), ("uidx", 4 * nnz, np.int32),
                           ("lcol", 2 * nnz, np.uint16)):
        out[name] = raw[o:o + size].view(dt)
        o += a16(size)
    o = (o + 31) // 32 * 32
    out["geo"] = raw[o:o + 16 * nt * 128 * maxrow].view(np.float32).reshape(-1, 4)
    o += 16 * nt * 128 * maxrow
    out["slots"] = raw[o:o + 2 * nt * 128 * maxrow].view(np.uint16)     # the TL plan's slot section
    o += a16(2 * nt * 128 * maxrow)
    out["wsum"] = raw[o:o + 16 * n].view(np.float32).reshape(n, 4)      # (S_i, 0) per particle
    o += a16(16 * n)
    out["spos"] = raw[o:o + 2 * nnz].view(np.uint16)                      # staging position per distinct neighbour
    o += a16(2 * nnz)
    out["sinv"] = raw[o:o + 2 * nnz].view(np.uint16)                      # its inverse
    return out


def _quarter_loads(slots):
    """Per quarter warp (8 consecutive rows), the largest number of its pairs in one group
    (position mod 8), summed over the tile's quarter warps."""
    tot = 0
    for q0 in range(0, len(slots), 8):
        allp = np.concatenate([np.asarray(sl) % 8 for sl in slots[q0:q0 + 8]]) if slots[q0:q0 + 8] else []
        if len(allp):
            tot += np.bincount(allp, minlength=8).max()
    return tot


def test_tile_plan_is_exact(ctx):
    # per tile of 128 rows: the ascending distinct columns, each pair's index among
    # them and the sliced pair factors w_ij = grad0 W_ij V0_j, against numpy on the
    # same lists (w in float64 by the oracle's kernel, rounded to float32 on the GPU)
    s = _setup(ctx, dp=0.004)
    n = s["r0"].shape[1]
    rp, col = host(s["rp"]), host(s["col"])           # the lists the plan was built from
    lens = np.diff(rp)
    sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    P = _read_plan(sol.plan, n, col.size, int(lens.max()))
    hdr = P["hdr"]
    assert (sol.st.plan_maxm, sol.st.plan_maxrow, sol.st.plan_nnz) == (hdr[0], hdr[2], col.size)
    dom = s["prm"].dom
    h = dom.h
    from oracle import kernels as OKer
    ms, ps = [], []
    # S_i = sum_j grad0 W_ij V0_j of every row (the geometry form's M_i half of Eq. 30)
    ii = np.repeat(np.arange(n), np.diff(rp))
    dxa = ON.min_image(s["r0"][:, ii] - s["r0"][:, col], dom)
    ra = np.sqrt(np.sum(dxa * dxa, axis=0))
    wa = OKer.wendland_dwdr(ra, h, 3, None) / ra * s["vol"][col] * dxa
    S = np.stack([np.bincount(ii, weights=wa[a], minlength=n) for a in range(3)])
    scale = np.abs(wa).max()
    assert np.allclose(P["wsum"][:, :3].T, S, rtol=2e-6, atol=1e-6 * scale)
    assert np.all(P["wsum"][:, 3] == 0.0)
    for b in range((n + 127) // 128):
        i0, i1 = 128 * b, min(n, 128 * b + 128)
        p0, p1 = rp[i0], rp[i1]
        u = np.unique(col[p0:p1])
        assert P["tile_m"][b] == u.size
        assert np.array_equal(P["uidx"][p0:p0 + u.size], u)
        lc = np.searchsorted(u, col[p0:p1])
        assert np.array_equal(P["lcol"][p0:p1], lc)
        width = int(lens[i0:i1].max())
        assert P["tile_e"][b] == 128 * width
        so = P["tile_so"][b]
        assert P["tile_so"][b + 1] == so + 128 * width
        # staging positions: a permutation of the tile's distinct neighbours, sinv its inverse
        spos = P["spos"][p0:p0 + u.size].astype(np.int64)
        assert np.array_equal(np.sort(spos), np.arange(u.size))
        assert np.array_equal(P["sinv"][p0 + spos], np.arange(u.size))
        lists = [lc[rp[i] - p0:rp[i + 1] - p0] for i in range(i0, i1)]
        slots = [spos[x] for x in lists]
        if b < 40:
            # the positions balance each quarter warp's pairs over the 8 groups at least as
            # well as the list order does
            assert _quarter_loads(slots) <= _quarter_loads(lists)
        orders = _match_order(slots) if b < 12 else None
        for r in range(i1 - i0):
            i = i0 + r
            k = np.arange(lens[i])
            ent = P["geo"][so + k * 128 + r]
            j = col[rp[i]:rp[i + 1]]
            dx = ON.min_image(s["r0"][:, i:i + 1] - s["r0"][:, j], dom)
            q = np.sqrt(np.sum(dx * dx, axis=0)) / h
            w = OKer.wendland_dwdr(q * h, h, 3, None) / (q * h) * s["vol"][j] * dx
            # the entries are the row's pairs, each once: the slot says which
            got = ent[:, 3].view(np.int32)
            o = np.array([np.flatnonzero(lists[r] == g)[0] for g in got], dtype=np.int64)
            assert np.array_equal(np.sort(o), k)
            if orders is not None:
                assert np.array_equal(o, orders[r])
            assert np.allclose(ent[:, :3].T, w[:, o], rtol=2e-6, atol=1e-6 * np.abs(w).max())
            pad = P["geo"][so + np.arange(lens[i], width) * 128 + r]
            assert np.all(pad == 0.0)
            # the slot section holds the entries' staging positions in the same sliced order
            assert np.array_equal(P["slots"][so + k * 128 + r], spos[got].astype(np.uint16))
        ms.append(u.size)
        ps.append(p1 - p0)
    assert hdr[0] == max(ms) and hdr[1] == max(ps) and hdr[2] == lens.max()
    # Morton order makes tiles compact: each tile's distinct neighbours are a few times its rows
    assert np.mean(ms) < 8 * 128


@pytest.mark.parametrize("dp", [0.005, 0.002])
def test_planned_pass_forms_agree_bitwise(ctx, dp):
    # the persistent, the streaming and the bulk-copy forms, each with its neighbours
    # staged in shared memory or (tiles over the stage capacity) read from global
    # memory: the same arithmetic in the same order
    s = _setup(ctx, dp=dp)
    ref = None
    for pipe in (api.SPH_PIPE_PERSISTENT, api.SPH_PIPE_STREAM, api.SPH_PIPE_BULK):
        for cap in (0, 16):
            ctx.set_tile_pipeline(pipe)
            ctx.set_stage_cap(cap)
            sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
            sol.step(3)
            a, F = sol.rates()
            x, v, H = sol.fields()
            got = [sol.rd.clone(), sol.rm.clone(), sol.H32.clone(), a, F]
            if ref is None:
                ref = got
            else:
                assert all(torch.equal(p, q) for p, q in zip(got, ref)), (pipe, cap)
    ctx.set_tile_pipeline(api.SPH_PIPE_GEOM)
    ctx.set_stage_cap(0)


def test_geometry_form_against_the_entry_form(ctx):
    # SPH_PIPE_GEOM evaluates grad0 W_ij V0_j in float32 where the entries hold it
    # rounded from float64, in the same pair order: the two agree to float32 rounding,
    # and so does the geometry form with its neighbours read from global memory (stage
    # capacity 16: the pair offsets from the cell codes instead of tile-relative positions)
    s = _setup(ctx, dp=0.004)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(3)
    H = 0.01 * rng.normal(size=(9, n))
    v = s["v"] + 0.1 * rng.normal(size=s["v"].shape)
    out = {}
    for pipe, cap in ((api.SPH_PIPE_STREAM, 0), (api.SPH_PIPE_GEOM, 0), (api.SPH_PIPE_GEOM, 16)):
        ctx.set_tile_pipeline(pipe)
        ctx.set_stage_cap(cap)
        try:
            sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN, v=v, H=H)
            a, Fd = sol.rates()
            sol.step(3)
            out[(pipe, cap)] = [a, Fd] + list(sol.fields())
        finally:
            ctx.set_stage_cap(0)
    ref, geo, glob = out[(api.SPH_PIPE_STREAM, 0)], out[(api.SPH_PIPE_GEOM, 0)], out[(api.SPH_PIPE_GEOM, 16)]
    for p, q, r in zip(geo[:2], ref[:2], glob[:2]):
        assert rel_l2(host(p), host(q)) < 1e-6 and rel_l2(host(r), host(q)) < 1e-6


def _dense_random_solid(n=1500, seed=3):
    """Random points in the unit cube with about 170 neighbours per interior particle at
    kappa = 1.6: rows longer than the 128 pairs the plan's ordering and the shared-memory
    slot block handle, so the list-order and global-slot fallbacks run."""
    rng = np.random.default_rng(seed)
    r0 = rng.uniform(0.0, 1.0, size=(3, n))
    h = 0.1875
    d = inputs.domain(3, h, 1.6, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0), (False, False, False))
    fixed = (r0[0] < 0.1).astype(np.uint8)
    v = 0.01 * rng.normal(size=(3, n))
    v[:, fixed == 1] = 0.0
    rho0, E, nu = 1000.0, 2.0e6, 0.3
    lam, G = E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))
    c0 = np.sqrt((lam + 2 * G) / rho0)
    return {"r0": r0, "v": v, "fixed": fixed, "vol": np.full(n, 1.0 / n), "domain": d, "dt": 0.1 * h / c0,
            "rho0": rho0, "lam": lam, "G": G}


def test_long_rows_against_the_oracle(ctx):
    # rows above 128 pairs: every float32 form, 3 steps, against the oracle
    case = _dense_random_solid()
    s = _setup(ctx, case=case)
    n = s["r0"].shape[1]
    assert np.max(np.diff(host(s["rp"]))) > 128
    F0 = np.tile(np.eye(3), (n, 1, 1))
    x_o, v_o, F_o = OT.run(s["r0"], s["vol"], s["B0_h"], s["fixed"], s["r0"].copy(), s["v"], F0, s["rp_h"],
                           s["col_h"], s["prm"], 3)
    H_o = (F_o - np.eye(3)[None]).reshape(n, 9).T
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN, tiles=tiles)
        sol.step(3)
        x, v, H = sol.fields()
        assert err(host(v), v_o) < tol, (prec, tiles, err(host(v), v_o))
        assert err(host(H), H_o) < tol, (prec, tiles, err(host(H), H_o))


@pytest.mark.parametrize("law", [OT.SVK, OT.NEO_HOOKEAN])
def test_energy_against_the_oracle(ctx, law):
    # kinetic and stored energy of a strained, moving state: float64 reduction at 1e-12
    s = _setup(ctx, law=law)
    n = s["r0"].shape[1]
    rng = np.random.default_rng(4)
    H = 0.02 * rng.normal(size=(9, n))
    v = s["v"] + 0.1 * rng.normal(size=s["v"].shape)
    ke_o, pe_o = OT.energies(s["r0"], s["vol"], v, _F_from_H(H), s["prm"])
    sol = _solid(ctx, s, api.SPH_FP64, law, v=v, H=H)
    ke, pe = sol.energy()
    assert abs(ke - ke_o) <= 1e-12 * ke_o and abs(pe - pe_o) <= 1e-12 * pe_o
    # a few steps later the float32 form's energy (read through its float64 unpack) stays
    # within float32 accuracy of the float64 run's
    a = _solid(ctx, s, api.SPH_FP64, law)
    b = _solid(ctx, s, api.SPH_FP32_KAHAN, law)
    a.step(20)
    b.step(20)
    ea, eb = a.energy(), b.energy()
    assert abs(sum(ea) - sum(eb)) <= 1e-5 * sum(ea)


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
    # the oracle's list and B0 on the sampled rows and their neighbours
    rp_o, col_o, B0_o, nb = oracle_rows(s["r0"], s["vol"], s["prm"].dom, rows, 1)
    Fm = np.tile(np.eye(3), (n, 1, 1))
    Fm[nb] = _F_from_H(H[:, nb])
    M = np.zeros((n, 3, 3))
    M[nb] = OT.stress_matrix(Fm[nb], B0_o[:, nb], s["prm"])
    rp_s, col_s = sample_rows(rp_o, col_o, rows)
    a_o = OT.momentum_rate(s["r0"], s["vol"], M, rp_s, col_s, s["prm"].dom, s["prm"].rho0)
    Fd_o = OT.deformation_rate(s["r0"], s["vol"], s["v"], B0_o, rp_s, col_s, s["prm"].dom).reshape(n, 9).T
    assert rel_l2(a[:, rows], a_o[:, rows]) < 1e-5
    assert rel_l2(Fd[:, rows], Fd_o[:, rows]) < 1e-5


def test_state_in_mapped_host_memory(ctx):
    # the float64 state (x, v, F - I) in mapped page-locked host buffers, read and
    # written in place by pack and unpack: the same results, bit for bit, as the
    # state in device memory
    s = _setup(ctx, dp=0.005)
    ref = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    mapped = [api.HostArray(t.shape) for t in (sol.x, sol.v, sol.H)]
    try:
        for m, t in zip(mapped, (sol.x, sol.v, sol.H)):
            m.t.copy_(t.cpu())
        sol.st.x, sol.st.v, sol.st.H = mapped[0].dev, mapped[1].dev, mapped[2].dev
        for _ in range(3):
            sol.pack()
            sol.step(2)
            sol.unpack()
            ref.pack()
            ref.step(2)
            ref.unpack()
        torch.cuda.synchronize()
        for m, t in zip(mapped, (ref.x, ref.v, ref.H)):
            assert torch.equal(m.t, t.cpu())
    finally:
        for m in mapped:
            m.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_step_host32_equals_the_composed_calls(ctx, dim):
    # sph_tlsph_step_host32 (copies overlapped with the passes on a second stream) gives
    # the state of load32 / step(1) / store32 in turn, bit for bit, in mapped host memory
    s = _setup(ctx, dp=0.005) if dim == 3 else _setup(ctx, case=inputs.beam2d(dp=0.002))
    n = s["r0"].shape[1]
    a = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    b = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    shapes = ((dim, n), (dim, n), (dim * dim, n))
    ha = [api.HostArray(sh, torch.float32) for sh in shapes]
    hb = [api.HostArray(sh, torch.float32) for sh in shapes]
    try:
        a.pack()
        b.pack()
        a.store32(*ha)
        b.store32(*hb)
        torch.cuda.synchronize()
        for _ in range(4):
            a.load32(*ha)
            a.step(1)
            a.store32(*ha)
        b.step_host32(*hb, nsteps=4)
        torch.cuda.synchronize()
        for x, y in zip(ha, hb):
            assert torch.equal(x.t, y.t)
        assert torch.equal(a.rd, b.rd) and torch.equal(a.H32, b.H32) and torch.equal(a.u32, b.u32)
        assert bool(torch.isfinite(hb[1].t).all()) and float(hb[1].t.abs().max()) > 0.0
        # on device arrays too
        dev = [torch.empty(sh, dtype=torch.float32, device="cuda") for sh in shapes]
        a.store32(*dev)
        a.step_host32(*dev, nsteps=2)
        b.step_host32(*hb, nsteps=2)
        torch.cuda.synchronize()
        for x, y in zip(dev, hb):
            assert torch.equal(x.cpu(), y.t)
    finally:
        for h in ha + hb:
            h.close()


@pytest.mark.parametrize("dim", [3, 2])
def test_l2_persistence_changes_nothing(ctx, dim):
    # the access-policy windows of the geometry-form passes (sph_set_l2_persist, on by
    # default) change only where the gathered records are cached: 10 steps with and without
    # them give the same records bit for bit; off gives the set-aside back, and the setting
    # takes only 0 or 1
    s = _setup(ctx, dp=0.005) if dim == 3 else _setup(ctx, case=inputs.beam2d(dp=0.002))
    a = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    b = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    try:
        ctx.set_l2_persist(True)
        a.step(10)
        torch.cuda.synchronize()
        ctx.set_l2_persist(False)
        b.step(10)
        torch.cuda.synchronize()
        for x, y in ((a.rd, b.rd), (a.rm, b.rm), (a.H32, b.H32), (a.u32, b.u32)):
            assert torch.equal(x, y)
        assert float(a.rd.abs().max()) > 0.0
        assert ctx.lib.sph_set_l2_persist(ctx.h, 2) == _lib.SPH_ERR_ARG
        assert ctx.lib.sph_set_l2_persist(None, 1) == _lib.SPH_ERR_ARG
    finally:
        ctx.set_l2_persist(True)


@pytest.mark.parametrize("dim", [3, 2])
def test_float32_state_round_trip(ctx, dim):
    # the float32 form's state kept in mapped host memory as float32 (u = x - r0, v, F - I)
    # and exchanged every 2 steps with load32 / store32: bit for bit the device-resident run;
    # and the float64 unpack of the same state agrees with it.  3D plate and 2D strip (the
    # 2D records keep v and the 2 x 2 H at other offsets)
    s = _setup(ctx, dp=0.005) if dim == 3 else _setup(ctx, case=inputs.beam2d(dp=0.002))
    n = s["r0"].shape[1]
    ref = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    bufs = [api.HostArray((dim, n), torch.float32), api.HostArray((dim, n), torch.float32),
            api.HostArray((dim * dim, n), torch.float32)]
    # the binding refuses buffers the C side would misread
    wrong = api.HostArray((dim, n))                      # float64
    try:
        with pytest.raises(ValueError):
            sol.store32(wrong, bufs[1], bufs[2])
        with pytest.raises(ValueError):
            sol.load32(bufs[0], bufs[1], torch.zeros((dim * dim, n), dtype=torch.float32, device="cuda").t())
    finally:
        wrong.close()
    try:
        ref.pack()
        sol.pack()
        sol.store32(*bufs)
        for _ in range(3):
            sol.load32(*bufs)
            sol.step(2)
            sol.store32(*bufs)
            ref.step(2)
        dev = [torch.empty((dim, n), dtype=torch.float32, device="cuda"),
               torch.empty((dim, n), dtype=torch.float32, device="cuda"),
               torch.empty((dim * dim, n), dtype=torch.float32, device="cuda")]
        ref.store32(*dev)
        torch.cuda.synchronize()
        for b, d in zip(bufs, dev):
            assert torch.equal(b.t, d.cpu())
        x, v, H = ref.fields()
        assert torch.equal(v.cpu().float(), bufs[1].t) and torch.equal(H.cpu().float(), bufs[2].t)
    finally:
        for b in bufs:
            b.close()


@pytest.mark.parametrize("kind", ["twisting", "bending"])
def test_columns_parity(ctx, kind):
    # the columns of Sec. 5 at side / dp = 4: float64 and float32 (tile plan and per pair)
    # against the oracle after 10 steps
    case = inputs.column(kind, 4)
    s = _setup(ctx, case=case)
    n = s["r0"].shape[1]
    x_o, v_o, F_o = s["r0"].copy(), s["v"].copy(), np.tile(np.eye(3), (n, 1, 1))
    for _ in range(10):
        x_o, v_o, F_o = OT.step(s["r0"], s["vol"], s["B0_h"], s["fixed"], x_o, v_o, F_o, s["rp_h"], s["col_h"],
                                s["prm"])
    H_o = (F_o - np.eye(3)).reshape(n, 9).T
    for prec, tiles, tol, err in VARIANTS:
        sol = _solid(ctx, s, prec, OT.NEO_HOOKEAN, tiles=tiles)
        sol.step(10)
        x, v, H = sol.fields()
        assert err(host(v), v_o) < tol, (prec, tiles, err(host(v), v_o))
        assert err(host(x) - s["r0"], x_o - s["r0"]) < tol
        assert err(host(H), H_o) < tol, (prec, tiles, err(host(H), H_o))


def test_sampled_kernel_timing(ctx):
    # events around every 3rd launch of each pass: 10 steps launch the stress once and
    # each pass 10 times; launches 1, 4, 7 and 10 of a pass are timed
    s = _setup(ctx, dp=0.005)
    sol = _solid(ctx, s, api.SPH_FP32_KAHAN, OT.NEO_HOOKEAN)
    ctx.timing(True, every=3)
    try:
        sol.step(10)
        counts = {k: ctx.launches(k) for k in (api.L.SPH_TIMER_TL_STRESS, api.L.SPH_TIMER_TL_MOMENTUM,
                                               api.L.SPH_TIMER_TL_DEFORM)}
        timed = {k: ctx.timer(k) for k in counts}
    finally:
        ctx.timing(False)
    assert counts == {api.L.SPH_TIMER_TL_STRESS: 1, api.L.SPH_TIMER_TL_MOMENTUM: 10, api.L.SPH_TIMER_TL_DEFORM: 10}
    assert timed[api.L.SPH_TIMER_TL_STRESS][1] == 1
    assert timed[api.L.SPH_TIMER_TL_MOMENTUM][1] == 4 and timed[api.L.SPH_TIMER_TL_DEFORM][1] == 4
    assert all(ms > 0.0 for ms, _ in timed.values())
