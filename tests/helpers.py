"""Shared helpers of the GPU parity tests."""
import numpy as np
import torch

from oracle import kgc as OK
from oracle import neighbors as ON


def odom(d):
    """oracle Domain from an inputs-style dict."""
    return ON.Domain(d["dim"], d["h"], d["kappa"], d["lo"], d["len"], d["periodic"])


def cuda(x, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device="cuda")


def host(t):
    torch.cuda.synchronize()
    return t.detach().cpu().numpy()


def rel_max(a, ref):
    """Normwise max relative error: max|a - ref| / max|ref| (the float64 parity measure)."""
    den = np.max(np.abs(ref))
    return float(np.max(np.abs(a - ref)) / (den if den > 0 else 1.0))


def rel_elem(a, ref, floor=1e-3):
    """Element-wise relative error, each element against |ref| plus `floor` times the
    field's largest magnitude (entries that cancel to near zero keep an absolute bound)."""
    den = np.abs(ref) + floor * np.max(np.abs(ref))
    den = np.where(den > 0, den, 1.0)
    return float(np.max(np.abs(a - ref) / den))


def rel_fp64(a, ref):
    """The float64 parity measure: the normwise max relative error, and the element-wise one
    (rel_elem, 1e-3 floor) scaled by 1e-3, so that a 1e-12 bound also holds every element
    to 1e-9 of its own magnitude (fields evolved over tens of steps gather rounding from
    sums taken in another order)."""
    return max(rel_max(a, ref), 1e-3 * rel_elem(a, ref))


def rel_l2(a, ref):
    """Relative L2 error (Eq. 10 form), the float32 parity measure."""
    den = np.linalg.norm(ref)
    return float(np.linalg.norm(a - ref) / (den if den > 0 else 1.0))


def sample_rows(row_ptr, col, rows):
    """CSR with the given rows kept and every other row emptied (same n)."""
    n = row_ptr.shape[0] - 1
    keep = np.zeros(n, dtype=bool)
    keep[rows] = True
    lens = np.where(keep, np.diff(row_ptr), 0)
    rp = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=rp[1:])
    parts = [col[row_ptr[i]:row_ptr[i + 1]] for i in np.sort(rows)]
    c = np.concatenate(parts).astype(np.int32) if parts else np.zeros(0, np.int32)
    return rp, c


def sorted_by_cells(pos, d):
    """Positions reordered by (cell id, index): the layout the pair loops use."""
    order = ON.cell_order(pos, odom(d))
    return pos[:, order], order


class OracleLists(dict):
    """A test setup whose oracle-side neighbour list and correction matrices (``rp_h``,
    ``col_h`` and the key ``b_key``) the oracle builds from the setup's own positions, on
    first use, so that no oracle input comes from the device."""

    def __init__(self, pos_key, b_key, **kw):
        super().__init__(**kw)
        self._pos_key = pos_key
        self._b_key = b_key

    def __missing__(self, key):
        if key not in ("rp_h", "col_h", self._b_key):
            raise KeyError(key)
        od = self["prm"].dom
        pos = self[self._pos_key]
        rp, col = ON.neighbors_cells(pos, od)
        B, _ = OK.kgc(pos, self["vol"], rp, col, od)
        self.update({"rp_h": rp, "col_h": col, self._b_key: B})
        return self[key]


def oracle_rows(pos, vol, od, rows, hops):
    """The oracle's neighbour list and correction matrices on the rows within ``hops``
    neighbour hops of ``rows`` (every other row empty): what a sampled check of a large set
    needs.  Returns (row_ptr, col, B, those rows)."""
    level = np.unique(np.asarray(rows, dtype=np.int64))
    for _ in range(hops):
        _, col = ON.neighbors_cells(pos, od, rows=level)
        level = np.unique(np.concatenate([level, col.astype(np.int64)]))
    rp, col = ON.neighbors_cells(pos, od, rows=level)
    B, _ = OK.kgc(pos, vol, rp, col, od)
    return rp, col, B, level
