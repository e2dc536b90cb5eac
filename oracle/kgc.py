"""Kernel-gradient-correction matrices of the oracle (test infrastructure).

Eq. 9 (Sec. 2.3.2): B_i = -( sum_j r_ij (x) grad W_ij V_j )^-1.  It replaces the
kernel gradient by (B_i + B_j)/2 grad W_ij in the Eulerian update (Eq. 27,
Sec. 3.1.2) and multiplies the kernel gradient in the total-Lagrangian update
(Eqs. 30-31, Sec. 3.2), where it is taken in the reference configuration.

With grad W_ij = (dW/dr) r_ij / r the summand r_ij (x) grad W_ij is symmetric, so
B_i is symmetric.  The oracle forms the upper triangle A_ab (a <= b) as
-sum_j V_j r_ij[a] grad W_ij[b], summing j in CSR (ascending) order, and inverts
with the adjugate formula.  It stores the unique entries row by row:
2D (B00, B01, B11), 3D (B00, B01, B02, B11, B12, B22).

Readings (the paper is silent on them):
* the kernel and cut-off of B are those of the physics (the truncated gradient
  for kappa = 1.6);
* a particle whose A_i is not finite, has trace <= 0 or has
  det A <= 1e-8 (tr A / d)^d is left uncorrected (B_i = I) and flagged;
* a pair at zero distance contributes nothing (its direction is undefined).
"""
import numpy as np

from .kernels import kernel_dwdr, WENDLAND
from .neighbors import pair_geometry

SYM_INDEX = {2: [(0, 0), (0, 1), (1, 1)],
             3: [(0, 0), (0, 1), (0, 2), (1, 1), (1, 2), (2, 2)]}
DET_RATIO = 1e-8


def kernel_gradients(pos, row_ptr, col, dom, kind=WENDLAND):
    """(i, j, r_ij, r, grad W_ij) for every stored pair."""
    i, j, rij, r = pair_geometry(pos, row_ptr, col, dom)
    dw = kernel_dwdr(kind, r, dom.h, dom.dim, None)   # list membership is the support test
    with np.errstate(invalid="ignore", divide="ignore"):
        scale = np.where(r > 0.0, dw / r, 0.0)
    grad = rij * scale
    return i, j, rij, r, grad


def sym_to_full(Bs, dim):
    """(nsym, n) unique entries -> (n, dim, dim) symmetric matrices."""
    n = Bs.shape[1]
    B = np.zeros((n, dim, dim))
    for s, (a, b) in enumerate(SYM_INDEX[dim]):
        B[:, a, b] = Bs[s]
        B[:, b, a] = Bs[s]
    return B


def full_to_sym(B):
    dim = B.shape[1]
    return np.stack([B[:, a, b] for (a, b) in SYM_INDEX[dim]])


def correction_sums(pos, vol, row_ptr, col, dom, kind=WENDLAND):
    """A_i = -sum_j V_j r_ij (x) grad W_ij, unique entries (nsym, n)."""
    n = pos.shape[1]
    i, j, rij, r, grad = kernel_gradients(pos, row_ptr, col, dom, kind)
    vj = vol[j]
    A = np.zeros((len(SYM_INDEX[dom.dim]), n))
    for s, (a, b) in enumerate(SYM_INDEX[dom.dim]):
        A[s] = -np.bincount(i, weights=vj * rij[a] * grad[b], minlength=n)
    return A


def invert_sym(A, dim):
    """Adjugate inverse of symmetric 2x2 / 3x3 matrices given by unique entries.

    Returns (B unique entries, fallback flags uint8)."""
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        if dim == 2:
            a00, a01, a11 = A
            det = a00 * a11 - a01 * a01
            tr = a00 + a11
            B = np.stack([a11, -a01, a00]) / det
        else:
            a00, a01, a02, a11, a12, a22 = A
            c00 = a11 * a22 - a12 * a12
            c01 = a02 * a12 - a01 * a22
            c02 = a01 * a12 - a02 * a11
            c11 = a00 * a22 - a02 * a02
            c12 = a01 * a02 - a00 * a12
            c22 = a00 * a11 - a01 * a01
            det = a00 * c00 + a01 * c01 + a02 * c02
            tr = a00 + a11 + a22
            B = np.stack([c00, c01, c02, c11, c12, c22]) / det
        finite = np.all(np.isfinite(A), axis=0)
        ok = finite & (tr > 0.0) & (det > DET_RATIO * (tr / dim) ** dim)
    ident = np.array([1.0 if a == b else 0.0 for (a, b) in SYM_INDEX[dim]])[:, None]
    B = np.where(ok[None, :], B, ident)
    return B, (~ok).astype(np.uint8)


def kgc(pos, vol, row_ptr, col, dom, kind=WENDLAND):
    """Eq. 9: B_i (unique entries, shape (nsym, n)) and the fallback flags."""
    A = correction_sums(pos, vol, row_ptr, col, dom, kind)
    return invert_sym(A, dom.dim)
