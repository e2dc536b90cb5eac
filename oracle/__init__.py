"""FP64 CPU oracle for the truncated-Wendland SPH hot path (arXiv 2405.05155).

This package is TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference legs of ``bench.py`` may import it. The product
path (the CUDA library and its Python binding) never calls into it, and it never
calls into the product path: the two share no code. The only module both sides
use is the seeded input generator ``paper_2405_05155_gb300.inputs``, which holds
none of the method's arithmetic.

Every function is a plain, slow, step-by-step restatement of the paper in
float64 numpy, citing the section or equation it follows.  Conventions used
throughout (they follow from Eqs. 7, 9, 18, 30 and 31, see ``kernels``):

* positions and vector fields are SoA arrays of shape ``(dim, n)``;
* ``r_ij = r_i - r_j`` (minimum image on periodic axes), ``e_ij = r_ij / |r_ij|``;
* ``grad W_ij = (dW/dr)(|r_ij|) e_ij`` is the gradient with respect to ``r_i``;
* neighbour lists are CSR (``row_ptr`` int64 of length n+1, ``col`` int32),
  each row ascending in j, self excluded, membership ``d^2 <= (kappa h)^2``.

Modules
-------
kernels    Wendland C2 (Eq. 6, truncated at 1.6h or standard 2h) and
           Laguerre-Gauss (Eq. 8) values and radial derivatives.
neighbors  cell binning / ordering and CSR neighbour lists (compact support,
           Eq. 5), by brute force and by a cell list.
kgc        kernel-gradient-correction matrices B_i (Eq. 9).
eulerian   Riemann-based Eulerian weakly-compressible SPH (Eqs. 18, 22, 25-27).
tlsph      total-Lagrangian SPH for solids (Eqs. 28-31).
relax      Laguerre-Gauss particle relaxation (Eqs. 7-8) and its residual.
mlp        the learned relaxation proposal (features, 3x128 GELU MLP, Adam).
metrics    the L2 error norm of Eq. 10.
"""
