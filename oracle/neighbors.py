"""Neighbour sets of the oracle (test infrastructure, see ``oracle/__init__``).

The paper fixes the neighbour set through the compact condition (Eq. 5, Sec. 2.2):
W = 0 when |r| > kappa h, so particle j is a neighbour of i exactly when
|r_ij| <= kappa h; the cut-off kappa h (2h standard, 1.6h truncated, Sec. 2.3.1)
sets the neighbour count and with it the cost (Sec. 1, Sec. 2.3.1).

Readings used here (the paper does not discuss them):

* the distance test is on the squared distance, evaluated in float64 as
  ``((dx*dx) + dy*dy) + dz*dz`` with each product and sum rounded separately
  (no fused multiply-add), against ``(kappa*h) * (kappa*h)``;
* on a periodic axis of length L the minimum image is taken once:
  dx > L/2 -> dx - L, dx < -L/2 -> dx + L (the box must be at least 2 kappa h);
* the cell grid used to find candidates has ``n_k = max(1, floor(len_k / (kappa h)))``
  cells of size ``len_k / n_k`` per axis; cell coordinates are
  ``floor((x_k - lo_k) / size_k)``, wrapped modulo n_k on periodic axes and clamped
  to ``[0, n_k - 1]`` otherwise; the linear cell id is ``(c_z n_y + c_y) n_x + c_x``;
* a particle's own entry is excluded, rows are sorted ascending in j.
"""
import math

import numpy as np


class Domain:
    """Problem geometry: dimension, smoothing length, cut-off factor, box, periodicity."""

    def __init__(self, dim, h, kappa, lo, length, periodic):
        self.dim = int(dim)
        self.h = float(h)
        self.kappa = float(kappa)
        self.lo = np.array(lo, dtype=np.float64)[: self.dim]
        self.len = np.array(length, dtype=np.float64)[: self.dim]
        self.periodic = tuple(bool(p) for p in periodic)[: self.dim]
        for k in range(self.dim):
            # one minimum-image shift finds every neighbour only if the box spans two cut-offs
            if self.periodic[k] and self.len[k] < 2.0 * self.kappa * self.h:
                raise ValueError("periodic box %g on axis %d is below 2 kappa h = %g"
                                 % (self.len[k], k, 2.0 * self.kappa * self.h))

    @property
    def rc(self):
        return self.kappa * self.h

    @property
    def rc2(self):
        rc = self.kappa * self.h
        return rc * rc

    def with_kappa(self, kappa):
        return Domain(self.dim, self.h, kappa, self.lo, self.len, self.periodic)


def min_image(dx, dom):
    """Minimum-image pair vector on periodic axes (one shift by the box length)."""
    out = np.array(dx, dtype=np.float64, copy=True)
    for k in range(dom.dim):
        if dom.periodic[k]:
            L = dom.len[k]
            half = 0.5 * L
            ok = out[k]
            out[k] = np.where(ok > half, ok - L, np.where(ok < -half, ok + L, ok))
    return out


def squared_distance(dx):
    """Sum of squares in axis order, each operation rounded separately."""
    d2 = dx[0] * dx[0]
    for k in range(1, dx.shape[0]):
        d2 = d2 + dx[k] * dx[k]
    return d2


def cell_grid(dom):
    """Number of cells and cell size per axis (each cell edge >= kappa h)."""
    rc = dom.rc
    ncell = [max(1, int(math.floor(dom.len[k] / rc))) for k in range(dom.dim)]
    size = [dom.len[k] / ncell[k] for k in range(dom.dim)]
    return ncell, size


def cell_coords(pos, dom):
    ncell, size = cell_grid(dom)
    c = np.empty(pos.shape, dtype=np.int64)
    for k in range(dom.dim):
        ck = np.floor((pos[k] - dom.lo[k]) / size[k]).astype(np.int64)
        if dom.periodic[k]:
            ck = np.mod(ck, ncell[k])
        else:
            ck = np.clip(ck, 0, ncell[k] - 1)
        c[k] = ck
    return c


def linear_cell_id(c, ncell):
    lin = c[c.shape[0] - 1].copy()
    for k in range(c.shape[0] - 2, -1, -1):
        lin = lin * ncell[k] + c[k]
    return lin


def cell_ids(pos, dom):
    ncell, _ = cell_grid(dom)
    return linear_cell_id(cell_coords(pos, dom), ncell)


def morton_key(c, ncell):
    """Morton (Z-order) key of integer cell coordinates c [dim][m].

    Bit l of the coordinate on axis a is placed at the next free key position, level
    by level from the least significant bit, axes in order; an axis with
    b_a = ceil(log2 n_a) bits drops out once they are used (the reading of the
    Morton key of the cell sort, Sec. 2.3)."""
    c = np.asarray(c, dtype=np.int64)
    dim = c.shape[0]
    bits = [int(n - 1).bit_length() for n in ncell]
    key = np.zeros(c.shape[1], dtype=np.int64)
    at = 0
    for level in range(max(bits) if bits else 0):
        for a in range(dim):
            if level < bits[a]:
                key |= ((c[a] >> level) & 1) << at
                at += 1
    return key


def cell_order(pos, dom):
    """Permutation sorting particles by (Morton key of the cell, original index), stable."""
    ncell, _ = cell_grid(dom)
    keys = morton_key(cell_coords(pos, dom), ncell)
    return np.argsort(keys, kind="stable").astype(np.int64)


def _csr_from_pairs(i, j, n):
    o = np.lexsort((j, i))
    i = i[o]
    j = j[o]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(i, minlength=n), out=row_ptr[1:])
    return row_ptr, j.astype(np.int32)


def neighbors_bruteforce(pos, dom):
    """All pairs i != j with d^2 <= (kappa h)^2, by direct O(N^2) enumeration."""
    pos = np.asarray(pos, dtype=np.float64)
    n = pos.shape[1]
    ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    dx = min_image(pos[:, ii] - pos[:, jj], dom)
    d2 = squared_distance(dx)
    keep = (d2 <= dom.rc2) & (ii != jj)
    return _csr_from_pairs(ii[keep], jj[keep], n)


def _neighbour_cell_lists(c, ncell, periodic, dim):
    """Distinct neighbouring cell coordinates per axis: {c-1, c, c+1} wrapped or clipped."""
    per_axis = []
    for k in range(dim):
        cand = []
        for o in (-1, 0, 1):
            ck = c[k] + o
            if periodic[k]:
                ck = np.mod(ck, ncell[k])
            else:
                ck = np.clip(ck, 0, ncell[k] - 1)
            cand.append(ck)
        per_axis.append(cand)
    return per_axis


def neighbors_cells(pos, dom, chunk=4096, rows=None):
    """Same set as ``neighbors_bruteforce``, found through the cell list.  With ``rows``,
    only those rows are filled (the others are empty): a sample of a large set."""
    pos = np.asarray(pos, dtype=np.float64)
    dim = dom.dim
    n = pos.shape[1]
    ncell, _ = cell_grid(dom)
    ntot = int(np.prod(ncell))
    c = cell_coords(pos, dom)
    ids = linear_cell_id(c, ncell)
    order = np.argsort(ids, kind="stable")
    counts = np.bincount(ids, minlength=ntot)
    start = np.zeros(ntot + 1, dtype=np.int64)
    np.cumsum(counts, out=start[1:])
    rc2 = dom.rc2
    out_i = []
    out_j = []
    sel = np.arange(n) if rows is None else np.unique(np.asarray(rows, dtype=np.int64))
    for s in range(0, len(sel), chunk):
        idx = sel[s:s + chunk]
        cs = c[:, idx]
        per_axis = _neighbour_cell_lists(cs, ncell, dom.periodic, dim)
        # all 3^dim combinations of per-axis candidates, then drop duplicates
        combos = []
        for oz in range(3 if dim == 3 else 1):
            for oy in range(3):
                for ox in range(3):
                    cc = [per_axis[0][ox], per_axis[1][oy]]
                    if dim == 3:
                        cc.append(per_axis[2][oz])
                    combos.append(linear_cell_id(np.stack(cc), ncell))
        cells = np.stack(combos, axis=1)  # (m, 3^dim)
        owner = np.repeat(idx, cells.shape[1])
        key = np.unique(owner.astype(np.int64) * ntot + cells.ravel())
        owner = key // ntot
        cell = key % ntot
        lens = counts[cell]
        total = int(lens.sum())
        if total == 0:
            continue
        ci = np.repeat(owner, lens)
        base = np.repeat(start[cell], lens)
        within = np.arange(total) - np.repeat(np.cumsum(lens) - lens, lens)
        cj = order[base + within]
        dx = min_image(pos[:, ci] - pos[:, cj], dom)
        d2 = squared_distance(dx)
        keep = (d2 <= rc2) & (ci != cj)
        out_i.append(ci[keep])
        out_j.append(cj[keep])
    if out_i:
        i = np.concatenate(out_i)
        j = np.concatenate(out_j)
    else:
        i = np.zeros(0, dtype=np.int64)
        j = np.zeros(0, dtype=np.int64)
    return _csr_from_pairs(i, j, n)


def pair_index(row_ptr, col):
    """Expand CSR into (i, j) arrays in row order."""
    n = row_ptr.shape[0] - 1
    i = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    return i, col.astype(np.int64)


def pair_geometry(pos, row_ptr, col, dom):
    """r_ij = r_i - r_j (minimum image), |r_ij| for every stored pair."""
    i, j = pair_index(row_ptr, col)
    rij = min_image(pos[:, i] - pos[:, j], dom)
    r = np.sqrt(squared_distance(rij))
    return i, j, rij, r
