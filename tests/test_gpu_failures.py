"""Failure detection on the GPU, in forms that fault and hang nothing.

A bounded device wait that runs out must surface as SPH_ERR_TIMEOUT on the host, with
the context still usable afterwards; a non-finite value met by a float64 reduction must
surface as SPH_ERR_NONFINITE, and a non-finite position as SPH_ERR_ARG.  The timeout is
provoked with the library's wait test (sph_set_wait_test): the TMA copies of the
bulk-copy and geometry-form deformation passes and of the planned Eulerian passes are then
not issued, so their bounded waits poll mbarrier phases that nothing completes, run out
after a few hundred polls, and every block leaves through the timeout branch with nothing
in flight.
"""
import numpy as np
import pytest
import torch

from helpers import cuda, host, sorted_by_cells
from paper_2405_05155_gb300 import _lib as L
from paper_2405_05155_gb300 import api, inputs, learned

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.set_wait_test(0)
    c.set_tile_pipeline(api.SPH_PIPE_GEOM)
    c.set_entry_ring(api.SPH_RING_AUTO)
    c.close()


def _plate_solid(ctx):
    c = inputs.plate(dp=0.005, kappa=1.6)
    d = c["domain"]
    r0, order = sorted_by_cells(c["r0"], d)
    rp, col = api.build_neighbors(ctx, d, cuda(r0))
    vol = c["vol"][order]
    B0, _, _ = api.kgc(ctx, d, cuda(r0), cuda(vol), rp, col)
    return api.TLSolid(ctx, d, cuda(r0), cuda(vol), B0, c["fixed"][order], rp, col, c["v"][:, order], c["dt"],
                       c["rho0"], c["lam"], c["G"], law=api.SPH_NEO_HOOKEAN, precision=api.SPH_FP32_KAHAN,
                       tiles=True)


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(ctx):
    ctx.set_tile_pipeline(api.SPH_PIPE_BULK)
    try:
        sol = _plate_solid(ctx)
        ctx.set_wait_test(256)
        try:
            sol.step(1)
            with pytest.raises(L.SphError) as e:
                sol.unpack()
            assert e.value.status == L.SPH_ERR_TIMEOUT
        finally:
            ctx.set_wait_test(0)
        # the flag was read and cleared: a normal run in the same context is clean and
        # equals the streamed form bit for bit (the bulk form's arithmetic is the same)
        sol = _plate_solid(ctx)
        sol.step(3)
        sol.unpack()
        ref_v = sol.v.clone()
        ctx.set_tile_pipeline(api.SPH_PIPE_STREAM)
        ref = _plate_solid(ctx)
        ref.step(3)
        ref.unpack()
        torch.cuda.synchronize()
        assert torch.isfinite(ref_v).all()
        assert torch.equal(ref_v, ref.v)
    finally:
        ctx.set_tile_pipeline(api.SPH_PIPE_GEOM)


def test_geometry_form_slot_copy_timeout_is_reported(ctx):
    # the default (geometry-form) deformation pass copies each tile's slot block with one
    # TMA bulk copy whose wait is bounded: under the wait test nothing is copied, the wait
    # runs out, the step reports SPH_ERR_TIMEOUT, and the same context then runs as before
    ctx.set_tile_pipeline(api.SPH_PIPE_GEOM)
    ref = _plate_solid(ctx)
    ref.step(2)
    ref.unpack()
    sol = _plate_solid(ctx)
    ctx.set_wait_test(256)
    try:
        sol.step(1)
        with pytest.raises(L.SphError) as e:
            sol.unpack()
        assert e.value.status == L.SPH_ERR_TIMEOUT
    finally:
        ctx.set_wait_test(0)
    again = _plate_solid(ctx)
    again.step(2)
    again.unpack()
    torch.cuda.synchronize()
    assert torch.isfinite(again.v).all() and torch.equal(again.v, ref.v)


def _tgv_sim(ctx):
    c = inputs.tgv3d(n=12, kappa=1.6)
    d = c["domain"]
    pos, order = sorted_by_cells(c["pos"], d)
    pos = cuda(pos)
    vol = cuda(c["vol"][order])
    rp, col = api.build_neighbors(ctx, d, pos)
    B, _, _ = api.kgc(ctx, d, pos, vol, rp, col)
    drho = api.density_from_pressure(ctx, d, c["c0"], cuda(c["p"][order]))
    return api.Eulerian(ctx, d, pos, vol, B, rp, col, drho, c["v"][:, order], c["dt"], c["rho0"], c["c0"], c["mu"],
                        precision=api.SPH_FP32_KAHAN, tiles=True)


def test_eulerian_entry_ring_timeout_is_reported(ctx):
    # the planned Eulerian passes take their pair entries through a ring of TMA bulk copies
    # with bounded waits: under the wait test nothing is copied, the waits run out, the
    # unpack reports SPH_ERR_TIMEOUT, and the same context then runs as before
    ctx.set_entry_ring(api.SPH_RING_CHUNK)
    try:
        ref = _tgv_sim(ctx)
        ref.step(2)
        ref.unpack()
        sim = _tgv_sim(ctx)
        ctx.set_wait_test(256)
        try:
            sim.step(1)
            with pytest.raises(L.SphError) as e:
                sim.unpack()
            assert e.value.status == L.SPH_ERR_TIMEOUT
        finally:
            ctx.set_wait_test(0)
        again = _tgv_sim(ctx)
        again.step(2)
        again.unpack()
        torch.cuda.synchronize()
        assert torch.isfinite(again.v).all() and torch.equal(again.v, ref.v) and torch.equal(again.drho, ref.drho)
    finally:
        ctx.set_entry_ring(api.SPH_RING_AUTO)


def test_wait_test_argument_checks(ctx):
    with pytest.raises(L.SphError) as e:
        ctx.set_wait_test(1 << 20)
    assert e.value.status == L.SPH_ERR_ARG


def test_nonfinite_values_are_reported(ctx):
    b, prm, pos, vol = learned.body_on_device(ctx, 3, 1.0 / 24.0, precision=api.SPH_FP64)
    r_ok = api.relax_residual(ctx, prm, pos, vol)
    assert np.isfinite(r_ok[0]) and r_ok[2] > 0
    # a NaN volume reaches the residual's float64 reduction
    bad_vol = vol.clone()
    bad_vol[bad_vol.numel() // 2] = float("nan")
    with pytest.raises(L.SphError) as e:
        api.relax_residual(ctx, prm, pos, bad_vol)
    assert e.value.status == L.SPH_ERR_NONFINITE
    # a NaN position is refused when the cells are built
    bad_pos = pos.clone()
    bad_pos[0, 5] = float("nan")
    with pytest.raises(L.SphError) as e:
        api.relax_residual(ctx, prm, bad_pos, vol)
    assert e.value.status == L.SPH_ERR_ARG
    # and the context is clean afterwards
    assert api.relax_residual(ctx, prm, pos, vol) == r_ok
