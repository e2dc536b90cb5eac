"""Pins of the oracle's neighbour sets (compact support, Eq. 5; cut-offs of Sec. 2.3.1)."""
import itertools
import math

import numpy as np
import pytest

from oracle import neighbors as N
from paper_2405_05155_gb300 import inputs


def _random_case(seed, dim, kappa, n, periodic, box=1.0, h=0.05):
    rng = np.random.default_rng(seed)
    pos = rng.uniform(0.0, box, size=(dim, n))
    if not periodic:
        # a few particles outside the cell box exercise the clamped cells
        pos[:, : max(1, n // 50)] += rng.uniform(-0.3, 0.3, size=(dim, max(1, n // 50)))
    dom = N.Domain(dim, h, kappa, [0.0] * dim, [box] * dim, [periodic] * dim)
    return pos, dom


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kappa", [1.6, 2.0])
@pytest.mark.parametrize("periodic", [True, False])
def test_cell_list_equals_brute_force(dim, kappa, periodic):
    pos, dom = _random_case(11 + dim, dim, kappa, 700 if dim == 2 else 900, periodic)
    a = N.neighbors_bruteforce(pos, dom)
    b = N.neighbors_cells(pos, dom)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("periodic", [True, False])
def test_row_sample_equals_the_full_rows(periodic):
    pos, dom = _random_case(5, 3, 1.6, 900, periodic)
    rp, col = N.neighbors_cells(pos, dom)
    rows = np.random.default_rng(1).choice(900, 40, replace=False)
    srp, scol = N.neighbors_cells(pos, dom, chunk=7, rows=rows)
    lens = np.diff(srp)
    assert np.all(lens[np.setdiff1d(np.arange(900), rows)] == 0)
    for i in rows:
        assert np.array_equal(scol[srp[i]:srp[i + 1]], col[rp[i]:rp[i + 1]])


@pytest.mark.parametrize("box_cells", [2, 3])
def test_few_cells_periodic_no_duplicates(box_cells):
    # box of exactly 2 or 3 cells per axis: c-1 and c+1 can be the same cell
    h = 0.1
    kappa = 2.0
    box = box_cells * kappa * h + 1e-9
    rng = np.random.default_rng(5)
    pos = rng.uniform(0.0, box, size=(2, 300))
    dom = N.Domain(2, h, kappa, [0.0, 0.0], [box, box], [True, True])
    a = N.neighbors_bruteforce(pos, dom)
    b = N.neighbors_cells(pos, dom)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _lattice_count(dim, h_over_dp, kappa):
    """Integer vectors k != 0 with |k| dp <= kappa h: pure enumeration, independent of the oracle."""
    rc = kappa * h_over_dp
    m = int(math.ceil(rc)) + 1
    c = 0
    for k in itertools.product(range(-m, m + 1), repeat=dim):
        s = sum(x * x for x in k)
        if s and s <= rc * rc:
            c += 1
    return c


@pytest.mark.parametrize("dim,h_over_dp,kappa,expected", [
    (2, 1.3, 1.6, 12), (2, 1.3, 2.0, 20), (3, 1.3, 1.6, 32), (3, 1.3, 2.0, 80),
    (3, 1.15, 1.6, 26), (3, 1.15, 2.0, 56)])
def test_lattice_neighbour_counts(dim, h_over_dp, kappa, expected):
    assert _lattice_count(dim, h_over_dp, kappa) == expected
    nx = 9
    dp = 1.0 / nx
    pos = inputs.lattice((nx,) * dim, dp)
    dom = N.Domain(dim, h_over_dp * dp, kappa, [0.0] * dim, [1.0] * dim, [True] * dim)
    rp, col = N.neighbors_cells(pos, dom)
    assert np.all(np.diff(rp) == expected)


def test_symmetry_sorted_rows_and_no_self():
    pos, dom = _random_case(3, 3, 1.6, 1500, True)
    rp, col = N.neighbors_cells(pos, dom)
    n = pos.shape[1]
    pairs = set()
    for i in range(n):
        row = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert i not in row
        pairs.update((i, int(j)) for j in row)
    assert all((j, i) in pairs for (i, j) in pairs)


def test_boundary_is_inclusive():
    # pair at exactly kappa h is a neighbour (Eq. 5 removes only |r| > kappa h)
    h = 0.5
    dom = N.Domain(2, h, 2.0, [0.0, 0.0], [10.0, 10.0], [False, False])
    pos = np.array([[1.0, 2.0, 3.0 + 1e-15], [1.0, 1.0, 1.0]])
    rp, col = N.neighbors_bruteforce(pos, dom)
    assert list(col[rp[0]:rp[1]]) == [1]
    assert list(col[rp[1]:rp[2]]) == [0]     # 2 -> 3+1e-15 is just outside
    assert np.array_equal(N.neighbors_cells(pos, dom)[1], col)


def test_minimum_image_once():
    dom = N.Domain(1, 0.1, 2.0, [0.0], [1.0], [True])
    dx = np.array([[0.6, -0.6, 0.5, -0.5, 0.2]])
    out = N.min_image(dx, dom)
    # exactly half a box is left alone; beyond it one box length is added or removed
    assert np.array_equal(out[0], np.array([0.6 - 1.0, -0.6 + 1.0, 0.5, -0.5, 0.2]))


def test_cell_order_is_stable_sort_by_morton_key():
    pos, dom = _random_case(9, 3, 2.0, 2000, False)
    order = N.cell_order(pos, dom)
    ncell, _ = N.cell_grid(dom)
    keys = N.morton_key(N.cell_coords(pos, dom), ncell)[order]
    assert sorted(order.tolist()) == list(range(pos.shape[1]))
    assert np.all(np.diff(keys) >= 0)
    same = np.diff(keys) == 0
    assert np.all(np.diff(order)[same] > 0)
    # particles of one cell stay together: equal keys <=> equal cells
    ids = N.cell_ids(pos, dom)[order]
    assert np.array_equal(np.diff(keys) == 0, np.diff(ids) == 0)


def test_morton_key_is_the_z_order():
    # 4 x 4: the Z curve visits 2 x 2 quadrants in the order (x, y) = 00, 10, 01, 11,
    # recursively (x in the even bits, y in the odd bits of the key)
    z = [(0, 0), (1, 0), (0, 1), (1, 1), (2, 0), (3, 0), (2, 1), (3, 1),
         (0, 2), (1, 2), (0, 3), (1, 3), (2, 2), (3, 2), (2, 3), (3, 3)]
    c = np.array(z).T
    assert N.morton_key(c, [4, 4]).tolist() == list(range(16))
    # 2 x 2 x 2: key = x + 2 y + 4 z
    g = np.array([(x, y, zz) for zz in range(2) for y in range(2) for x in range(2)]).T
    assert N.morton_key(g, [2, 2, 2]).tolist() == list(range(8))
    # uneven axes (5 x 2 x 3 cells: 3, 1 and 2 bits): once y is used up the key
    # continues x, z, x; keys stay distinct and below 2^(3 + 1 + 2)
    g = np.array([(x, y, zz) for zz in range(3) for y in range(2) for x in range(5)]).T
    k = N.morton_key(g, [5, 2, 3])
    assert len(set(k.tolist())) == 30 and k.max() < 64
    for x, y, zz, kk in zip(g[0], g[1], g[2], k):
        expect = (x & 1) | (y & 1) << 1 | (zz & 1) << 2 | ((x >> 1) & 1) << 3 | ((zz >> 1) & 1) << 4 | ((x >> 2) & 1) << 5
        assert kk == expect
    # locality: in an 8^3 grid every aligned 2^3 block holds 8 consecutive keys
    g = np.array([(x, y, zz) for zz in range(8) for y in range(8) for x in range(8)]).T
    k = N.morton_key(g, [8, 8, 8])
    blocks = (g[0] // 2) + 4 * (g[1] // 2) + 16 * (g[2] // 2)
    for b in range(64):
        kb = np.sort(k[blocks == b])
        assert np.array_equal(kb, np.arange(kb[0], kb[0] + 8)) and kb[0] % 8 == 0
