"""SPH approximations of a field and of its gradient, oracle version (test infrastructure).

The error analysis of Sec. 2.3.3 measures, with the L2 error of Eq. 10:

* the kernel summation  f_i ~ sum_j f_j W_ij V_j,  j over the support of i including
  i itself; for f = 1 this is the normalisation condition of Eq. 3 (Table 1);
* the weak form of Eq. 4 for the gradient.  With grad W_ij = grad_i W (the
  convention under which Eqs. 7, 9, 18, 30 and 31 hold),
      grad f_i ~ sum_j (f_i + f_j) B_i grad W_ij V_j,
  with the correction matrix B_i of Eq. 9 ("with B") or B_i = I ("without B").

Pairs are those of the CSR lists with d^2 <= (kappa h)^2, as everywhere else.
"""
import numpy as np

from .kernels import WENDLAND, kernel_dwdr, kernel_w
from .kgc import sym_to_full
from .neighbors import pair_geometry, squared_distance


def kernel_sum(pos, vol, f, row_ptr, col, dom, kind=WENDLAND):
    """sum_j f_j W_ij V_j over the listed neighbours and i itself, shape (n,)."""
    n = pos.shape[1]
    i, j, rij, r = pair_geometry(pos, row_ptr, col, dom)
    within = squared_distance(rij) <= dom.rc2
    w = np.where(within, kernel_w(kind, r, dom.h, dom.dim, None), 0.0)
    s = np.bincount(i, weights=f[j] * w * vol[j], minlength=n)
    w0 = float(kernel_w(kind, 0.0, dom.h, dom.dim, None))
    return s + f * vol * w0


def weak_gradient(pos, vol, f, row_ptr, col, dom, B=None, kind=WENDLAND):
    """sum_j (f_i + f_j) B_i grad W_ij V_j (B = None: the identity), shape (dim, n).
    B holds the unique entries of the symmetric B_i, (dim (dim + 1) / 2, n)."""
    n, dim = pos.shape[1], dom.dim
    i, j, rij, r = pair_geometry(pos, row_ptr, col, dom)
    within = squared_distance(rij) <= dom.rc2
    dw = np.where(within, kernel_dwdr(kind, r, dom.h, dim, None), 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        g = np.where(r > 0.0, dw / r, 0.0) * rij               # grad_i W_ij, (dim, pairs)
    if B is not None:
        Bf = sym_to_full(np.asarray(B, dtype=np.float64), dim)  # (n, dim, dim)
        g = np.einsum("pab,bp->ap", Bf[i], g)
    c = (f[i] + f[j]) * vol[j]
    out = np.zeros((dim, n))
    for a in range(dim):
        out[a] = np.bincount(i, weights=c * g[a], minlength=n)
    return out
