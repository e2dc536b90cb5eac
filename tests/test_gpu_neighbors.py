"""GPU parity of a1 (cell order), a2 (CSR neighbour lists), a3 (kernel values) and a4 (KGC)
against the float64 oracle.  Neighbour lists and orders must be bit-exact."""
import ctypes

import numpy as np
import pytest
import torch

from helpers import cuda, host, odom, rel_fp64, rel_max, sample_rows, sorted_by_cells
from oracle import kernels as OKr
from oracle import kgc as OK
from oracle import neighbors as ON
from paper_2405_05155_gb300 import _lib, api, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = api.Context(0)
    yield c
    c.close()


def _random(seed, dim, kappa, n, periodic, box=1.0, h=0.04):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, size=(dim, n))
    if not periodic:
        pos[:, : n // 40] += rng.uniform(-0.3, 0.3, size=(dim, n // 40))
    d = inputs.domain(dim, h, kappa, [0.0] * dim, [box] * dim, [periodic] * dim)
    return pos, d


CASES = [(s, dim, kappa, per) for s, (dim, kappa, per) in enumerate(
    [(2, 1.6, True), (2, 2.0, False), (3, 1.6, False), (3, 2.0, True), (3, 1.6, True), (2, 1.6, False)])]


@pytest.mark.parametrize("seed,dim,kappa,periodic", CASES)
def test_neighbors_bit_exact_random(ctx, seed, dim, kappa, periodic):
    pos, d = _random(seed, dim, kappa, 3000 if dim == 2 else 6000, periodic)
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    rp_o, col_o = ON.neighbors_cells(pos, odom(d))
    assert np.array_equal(host(rp), rp_o)
    assert np.array_equal(host(col), col_o)


@pytest.mark.parametrize("which", ["tgv2d", "tgv3d", "plate", "body"])
def test_neighbors_bit_exact_workloads(ctx, which):
    if which == "tgv2d":
        c = inputs.tgv2d(nx=50)
        pos, d = c["pos"], c["domain"]
    elif which == "tgv3d":
        c = inputs.tgv3d(n=24, kappa=2.0)
        pos, d = c["pos"], c["domain"]
    elif which == "plate":
        c = inputs.plate(dp=0.004)
        pos, d = c["r0"], c["domain"]
    else:
        c = inputs.sphere_body(5, 1.0 / 32.0)
        pos, d = c["pos"], c["domain"]
    for p in (pos, sorted_by_cells(pos, d)[0]):
        rp, col = api.build_neighbors(ctx, d, cuda(p))
        rp_o, col_o = ON.neighbors_cells(p, odom(d))
        assert np.array_equal(host(rp), rp_o) and np.array_equal(host(col), col_o)


def test_lattice_distance_ties_and_boundary(ctx):
    # pairs at exactly kappa h (representable) are neighbours; one ulp further they are not
    h = 0.5
    pos = np.array([[1.0, 2.0, 3.0 + 2.0 ** -50, 5.0, 6.0], [1.0, 1.0, 1.0, 1.0, 1.0]])
    d = inputs.domain(2, h, 2.0, [0.0, 0.0], [8.0, 4.0], [False, False])
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    rp_o, col_o = ON.neighbors_bruteforce(pos, odom(d))
    assert np.array_equal(host(rp), rp_o) and np.array_equal(host(col), col_o)
    assert list(host(col)[host(rp)[0]:host(rp)[1]]) == [1]


def test_cell_order_bit_exact(ctx):
    for seed, dim, kappa, per in CASES:
        pos, d = _random(seed, dim, kappa, 4000, per)
        order = api.cell_order(ctx, d, cuda(pos))
        assert np.array_equal(host(order), ON.cell_order(pos, odom(d)))


def test_edge_cases(ctx):
    # empty input
    d = inputs.domain(3, 0.1, 2.0, [0, 0, 0], [1, 1, 1], [False] * 3)
    rp, col = api.build_neighbors(ctx, d, torch.zeros((3, 0), dtype=torch.float64, device="cuda"))
    assert host(rp).tolist() == [0] and col.numel() == 0
    # a single particle
    rp, col = api.build_neighbors(ctx, d, cuda(np.full((3, 1), 0.5)))
    assert host(rp).tolist() == [0, 0]
    # too small a capacity: the required size comes back, row_ptr is valid
    pos, d2 = _random(3, 2, 2.0, 500, True)
    dd = api.make_domain(d2, 500)
    rp = torch.empty(501, dtype=torch.int64, device="cuda")
    col = torch.empty(10, dtype=torch.int32, device="cuda")
    nnz = ctypes.c_int64()
    st = ctx.lib.sph_build_neighbors(ctx.h, ctypes.byref(dd), ctypes.c_void_p(cuda(pos).data_ptr()),
                                     ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(col.data_ptr()), 10,
                                     ctypes.byref(nnz), None)
    torch.cuda.synchronize()
    assert st == _lib.SPH_ERR_CAPACITY
    assert nnz.value == ON.neighbors_bruteforce(pos, odom(d2))[0][-1]
    # a position outside a periodic box and a NaN are reported, not computed on
    bad = pos.copy()
    bad[0, 7] = 1.5
    with pytest.raises(_lib.SphError):
        api.build_neighbors(ctx, d2, cuda(bad))
    bad = pos.copy()
    bad[1, 3] = np.nan
    with pytest.raises(_lib.SphError):
        api.build_neighbors(ctx, d2, cuda(bad))
    # the context still works afterwards
    rp, col = api.build_neighbors(ctx, d2, cuda(pos))
    assert np.array_equal(host(col), ON.neighbors_cells(pos, odom(d2))[1])


@pytest.mark.parametrize("kernel,kappa", [(api.SPH_WENDLAND_C2, 1.6), (api.SPH_WENDLAND_C2, 2.0),
                                          (api.SPH_LAGUERRE_GAUSS, 2.0)])
@pytest.mark.parametrize("dim", [2, 3])
def test_kernel_eval(kernel, kappa, dim):
    h = 0.037
    r = np.linspace(0.0, 2.1 * h, 5001)
    kind = OKr.WENDLAND if kernel == api.SPH_WENDLAND_C2 else OKr.LAGUERRE_GAUSS
    w_o = OKr.kernel_w(kind, r, h, dim, kappa)
    dw_o = OKr.kernel_dwdr(kind, r, h, dim, kappa)
    inside = r / h <= kappa * (1 - 1e-12)
    for prec, tol in ((api.SPH_FP64, 1e-14), (api.SPH_FP32_KAHAN, 2e-6)):
        w, dw = api.kernel_eval(kernel, dim, h, kappa, prec, cuda(r))
        w, dw = host(w), host(dw)
        assert rel_max(w[inside], w_o[inside]) < tol
        assert rel_max(dw[inside], dw_o[inside]) < tol
        assert np.all(w[r / h > kappa * (1 + 1e-6)] == 0.0)


@pytest.mark.parametrize("which", ["tgv2d", "tgv3d", "plate", "jitter2d"])
def test_kgc_parity(ctx, which):
    if which == "tgv2d":
        c = inputs.tgv2d(nx=40)
        pos, d, vol = c["pos"], c["domain"], c["vol"]
    elif which == "tgv3d":
        c = inputs.tgv3d(n=16)
        pos, d, vol = c["pos"], c["domain"], c["vol"]
    elif which == "plate":
        c = inputs.plate(dp=0.005)
        pos, d, vol = c["r0"], c["domain"], c["vol"]
    else:
        rng = np.random.default_rng(2)
        c = inputs.tgv2d(nx=40)
        d = c["domain"]
        pos = np.mod(c["pos"] + rng.uniform(-0.3, 0.3, c["pos"].shape) * c["dp"], 1.0)
        vol = c["vol"]
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    B, fb, nfb = api.kgc(ctx, d, cuda(pos), cuda(vol), rp, col)
    B_o, fb_o = OK.kgc(pos, vol, host(rp), host(col), odom(d))
    assert np.array_equal(host(fb), fb_o) and nfb == int(fb_o.sum())
    assert rel_fp64(host(B), B_o) < 1e-12


def test_kgc_fallback_and_lg_kernel(ctx):
    c = inputs.sphere_body(2, 1.0 / 24.0)
    pos, d, vol = c["pos"], dict(c["domain"]), c["vol"]
    pos = np.concatenate([pos, [[3.0], [3.0], [3.0]]], axis=1)          # an isolated particle
    vol = np.append(vol, vol[0])
    d["len"] = [4.0, 4.0, 4.0]
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    for kernel, kind in ((api.SPH_WENDLAND_C2, OKr.WENDLAND), (api.SPH_LAGUERRE_GAUSS, OKr.LAGUERRE_GAUSS)):
        B, fb, nfb = api.kgc(ctx, d, cuda(pos), cuda(vol), rp, col, kernel)
        B_o, fb_o = OK.kgc(pos, vol, host(rp), host(col), odom(d), kind)
        assert host(fb)[-1] == 1 and np.array_equal(host(fb), fb_o)
        assert rel_fp64(host(B), B_o) < 1e-12


def test_full_size_plate_neighbors_sampled(ctx):
    # the 0.2 x 0.02 x 0.2 m plate at dp = 1 mm (816k particles): sampled rows against brute force
    c = inputs.plate(dp=0.001)
    pos, d = c["r0"], c["domain"]
    rp, col = api.build_neighbors(ctx, d, cuda(pos))
    rp_h, col_h = host(rp), host(col)
    n = pos.shape[1]
    rng = np.random.default_rng(0)
    rows = rng.choice(n, 200, replace=False)
    dom = odom(d)
    for i in rows:
        dx = ON.min_image(pos[:, [i]] - pos, dom)
        d2 = ON.squared_distance(dx)
        expect = np.nonzero((d2 <= dom.rc2) & (np.arange(n) != i))[0]
        assert np.array_equal(col_h[rp_h[i]:rp_h[i + 1]], expect)
    # lattice interior rows have the 26 neighbours of h = 1.15 dp, kappa = 1.6
    assert np.max(np.diff(rp_h)) == 26
