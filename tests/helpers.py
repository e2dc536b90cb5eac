"""Shared helpers of the GPU parity tests."""
import numpy as np
import torch

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
