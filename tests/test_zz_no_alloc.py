"""The allocation-free neighbour build, sph_build_neighbors_static.

It exists for callers that cannot allocate device memory: a plug-in inside an
application that owns the device-memory budget and forbids any other cudaMalloc,
or a latency-critical loop in which cudaMalloc / cudaFree would synchronise the
device.  It must return exactly what sph_build_neighbors returns (neighbour lists
are integer results, compared bit for bit), on consecutive calls that share its
static scratch array, and it must reject inputs beyond its fixed limits.

This file is named so that pytest collects it last; it also passes when run on
its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2405_05155_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


def _static_call(lib, dom, pos, cap, free_delta=None):
    n = pos.shape[1]
    d = api.make_domain(dom, n)
    row_ptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
    col = torch.empty(max(cap, 1), dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64(-1)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    st = lib.sph_build_neighbors_static(ctypes.byref(d), ctypes.c_void_p(pos.data_ptr()),
                                        ctypes.c_void_p(row_ptr.data_ptr()), ctypes.c_void_p(col.data_ptr()),
                                        cap, ctypes.byref(nnz), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    if free_delta is not None:
        free_delta.append(free0 - torch.cuda.mem_get_info()[0])
    return st, row_ptr, col[: max(nnz.value, 0)], nnz.value


def _cases():
    # a dense 3D body first, then a smaller periodic 2D set: the second call must not see
    # anything left in the shared scratch by the first
    body = inputs.sphere_body(11, 1.0 / 48.0)
    rng = np.random.default_rng(4)
    pos2 = rng.uniform(0.0, 1.0, size=(2, 5000))
    dom2 = inputs.domain(2, 0.01, 1.6, [0.0, 0.0], [1.0, 1.0], [True, True])
    return [(body["domain"], body["pos"]), (dom2, pos2)]


def test_static_variant_matches_the_allocating_entry_point_on_consecutive_calls():
    lib = _lib.load()
    ctx = api.Context(0)
    try:
        for dom, pos_h in _cases():
            pos = torch.tensor(pos_h, dtype=torch.float64, device="cuda")
            rp_ref, col_ref = api.build_neighbors(ctx, dom, pos)
            nnz_ref = int(col_ref.numel())
            st, rp, col, nnz = _static_call(lib, dom, pos, nnz_ref)
            assert st == _lib.SPH_OK, lib.sph_status_string(st)
            assert nnz == nnz_ref
            assert torch.equal(rp, rp_ref)
            assert torch.equal(col, col_ref)
    finally:
        ctx.close()


def test_static_variant_repeats_without_allocating_and_rejects_oversized_input():
    lib = _lib.load()
    dom, pos_h = _cases()[0]
    pos = torch.tensor(pos_h, dtype=torch.float64, device="cuda")
    st, rp0, col0, nnz0 = _static_call(lib, dom, pos, 200 * pos.shape[1])
    assert st == _lib.SPH_OK
    delta = []
    st, rp1, col1, nnz1 = _static_call(lib, dom, pos, nnz0, free_delta=delta)
    assert st == _lib.SPH_OK and nnz1 == nnz0
    assert torch.equal(rp0, rp1) and torch.equal(col0, col1)
    # the call itself took no device memory (its outputs were allocated before it)
    assert delta[0] == 0
    # too small a column array: the required size comes back
    st, _, _, need = _static_call(lib, dom, pos, 10)
    assert st == _lib.SPH_ERR_CAPACITY and need == nnz0
    # more particles than the static array holds: rejected before any device work
    d = api.make_domain(dom, _lib.SPH_STATIC_MAX_PARTICLES + 1)
    nnz = ctypes.c_int64()
    st = lib.sph_build_neighbors_static(ctypes.byref(d), ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(1),
                                        ctypes.c_void_p(1), 0, ctypes.byref(nnz), None)
    assert st == _lib.SPH_ERR_LIMIT
    assert b"static scratch" in lib.sph_status_string(st)


def test_static_variant_against_the_oracle():
    # directly against the float64 oracle's cell-list build (itself pinned to brute force),
    # on a random 3D set in a closed box and a periodic 2D set, two calls in a row
    from oracle import neighbors as ON
    lib = _lib.load()
    rng = np.random.default_rng(9)
    pos3 = rng.uniform(0.0, 1.0, size=(3, 3000))
    dom3 = inputs.domain(3, 0.05, 1.6, [0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [False, False, False])
    pos2 = rng.uniform(0.0, 1.0, size=(2, 4000))
    dom2 = inputs.domain(2, 0.012, 2.0, [0.0, 0.0], [1.0, 1.0], [True, True])
    for dom, pos_h in ((dom3, pos3), (dom2, pos2)):
        od = ON.Domain(dom["dim"], dom["h"], dom["kappa"], dom["lo"], dom["len"], dom["periodic"])
        rp_o, col_o = ON.neighbors_cells(pos_h, od)
        pos = torch.tensor(pos_h, dtype=torch.float64, device="cuda")
        st, rp, col, nnz = _static_call(lib, dom, pos, int(col_o.size))
        assert st == _lib.SPH_OK, lib.sph_status_string(st)
        assert nnz == col_o.size
        assert np.array_equal(rp.cpu().numpy(), rp_o)
        assert np.array_equal(col.cpu().numpy(), col_o)
