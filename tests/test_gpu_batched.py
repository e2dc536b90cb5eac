"""GPU parity of the batched Eulerian step (a13): one persistent launch per pass over many
uneven cases must match each case run alone (to float32 rounding, same launch shape) and the
float64 oracle (float32 tolerance); the autotuner and the captured graph must not change it."""
import numpy as np
import pytest
import torch

from helpers import host, odom, rel_l2
from oracle import eulerian as OE
from oracle import kgc as OK
from oracle import neighbors as ON
from paper_2405_05155_gb300 import api, batch, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _small_cases():
    return inputs.batched_tgv2d(seed=3, ncases=7, scale=0.06)


@pytest.mark.parametrize("tiles,ring", [(True, api.SPH_RING_THREAD), (True, api.SPH_RING_CHUNK), (False, None)])
def test_batched_matches_single_case_runs(ctx, tiles, ring):
    # planned form (every case with a tile plan; the entries through the thread ring or the
    # TMA chunk ring, the same in both runs) or the persistent per-pair form
    if ring is not None:
        ctx.set_entry_ring(ring)
    cases = _small_cases()
    for lanes in (1, 4):
        ctx.set_lanes(api.SPH_PASS_EULERIAN, lanes)
        ctx.set_lanes(api.SPH_PASS_BATCHED, lanes)
        b = batch.EulerianBatch(ctx, cases, tiles=tiles)
        b.step(6)
        for c, sim in enumerate(b.sims):
            # the single-case path on the same initial packed state
            sim.pack()
            sim.step(6)
            torch.cuda.synchronize()
            single = sim.rec.clone()
            t = b.table[c]
            got = b.rec[16 * t.offset: 16 * (t.offset + t.n)]
            if tiles:
                # both run the planned tile body with explicit arithmetic: identical results
                assert torch.equal(got, single), c
            else:
                # same arithmetic per particle; the two kernels may contract a multiply-add differently
                assert rel_l2(host(got).astype(np.float64), host(single).astype(np.float64)) < 1e-6, c
    ctx.set_lanes(api.SPH_PASS_EULERIAN, 4)
    ctx.set_lanes(api.SPH_PASS_BATCHED, 4)
    ctx.set_entry_ring(api.SPH_RING_AUTO)


@pytest.mark.parametrize("tiles", [True, False])
def test_batched_against_oracle_and_autotune(ctx, tiles):
    cases = _small_cases()
    b = batch.EulerianBatch(ctx, cases, tiles=tiles)
    lanes, block, ms = b.autotune(trial_steps=3)
    assert lanes in (1, 2, 4, 8) and block in (128, 256) and ms > 0
    assert ctx.get_lanes(api.SPH_PASS_BATCHED) == lanes
    b.step(5)
    for c, case in enumerate(cases):
        d = case["domain"]
        dom = odom(d)
        order = ON.cell_order(case["pos"], dom)      # the layout the batch keeps its fields in
        assert np.array_equal(host(b.orders[c]), order)
        pos = case["pos"][:, order]
        rp, col = ON.neighbors_cells(pos, dom)
        vol = case["vol"][order]
        Bs, _ = OK.kgc(pos, vol, rp, col, dom)
        prm = OE.EulerianParams(dom, case["dt"], case["rho0"], case["c0"], case["mu"])
        d_o, v_o = OE.run(pos, vol, (case["p"] / case["c0"] ** 2)[order], case["v"][:, order], Bs, rp, col, prm, 5)
        dr, v = b.fields(c)
        assert rel_l2(host(dr), d_o) < 1e-5 and rel_l2(host(v), v_o) < 1e-5, c


def test_graph_is_recaptured_when_buffers_change(ctx):
    cases = _small_cases()[:3]
    b1 = batch.EulerianBatch(ctx, cases)
    b2 = batch.EulerianBatch(ctx, cases)
    b1.step(2)
    b2.step(1)
    b2.step(1)
    b1.step(1)
    b2.step(1)
    torch.cuda.synchronize()
    assert torch.equal(b1.rec, b2.rec)
