"""Kernel functions of the oracle (test infrastructure, see ``oracle/__init__``).

Wendland C2, Eq. 6 (Sec. 2.3.1).  The printed argument is garbled ("s <= kappa h"
with s = |r| while the polynomial is written in s/2); the only reading under which
the printed normalisation constants alpha_d normalise the polynomial is
q = r / h with support q <= kappa, and alpha_d carries the factor h^-d:

    W(r, h) = alpha_d h^-d (1 - q/2)^4 (2q + 1),   q = r/h <= kappa,
    alpha_1 = 3/4,  alpha_2 = 7/(4 pi),  alpha_3 = 21/(16 pi).

The truncated kernel (Sec. 2.3.1, "truncate the compact support from 2h to 1.6h")
is the same function cut at kappa = 1.6 without renormalisation; W and dW/dr are
exactly zero for q > kappa and the boundary q = kappa is inside (Eq. 5 sets W = 0
only for |r| > kappa h).

Inside the pair loops the support test is the neighbour-list predicate
d^2 <= (kappa h)^2 (see ``neighbors``); there the functions below are called with
``kappa=None`` (no second cut), so that the list alone decides membership and a
pair at q = kappa + 1 ulp after rounding is not dropped twice over.

Laguerre-Gauss, Eq. 8 (Sec. 2.3.2), support q <= 2:

    W(r, h) = ahat_d h^-d (1 - q^2/2 + q^4/6) exp(-q^2).

The printed alpha_d of Eq. 8 (8/(5 sqrt pi), 3/pi, 8/pi^1.5) do not normalise the
printed polynomial; the oracle uses the whole-space normalisation of that
polynomial, ahat_1 = 8/(7 sqrt pi), ahat_2 = 6/(5 pi), ahat_3 = 8/(7 pi^1.5).
Relaxation (Eq. 7 with the time step rule used here) is invariant to any
constant factor in the kernel, so this reading changes no particle position.
"""
import math

import numpy as np

ALPHA_WENDLAND = {1: 3.0 / 4.0, 2: 7.0 / (4.0 * math.pi), 3: 21.0 / (16.0 * math.pi)}
ALPHA_LG = {1: 8.0 / (7.0 * math.sqrt(math.pi)), 2: 6.0 / (5.0 * math.pi),
            3: 8.0 / (7.0 * math.pi ** 1.5)}
# The constants exactly as Eq. 8 prints them (kept for the test that shows
# they do not normalise the printed polynomial).
ALPHA_LG_PRINTED = {1: 8.0 / (5.0 * math.sqrt(math.pi)), 2: 3.0 / math.pi,
                    3: 8.0 / math.pi ** 1.5}

KAPPA_STANDARD = 2.0
KAPPA_TRUNCATED = 1.6
KAPPA_LG = 2.0

WENDLAND = "wendland"
LAGUERRE_GAUSS = "laguerre_gauss"


def wendland_w(r, h, dim, kappa):
    """Wendland C2 value W(r, h), Eq. 6, cut at q = kappa (kappa = 2 or 1.6)."""
    r = np.asarray(r, dtype=np.float64)
    q = r / h
    w = ALPHA_WENDLAND[dim] * h ** (-dim) * (1.0 - 0.5 * q) ** 4 * (2.0 * q + 1.0)
    return w if kappa is None else np.where(q <= kappa, w, 0.0)


def wendland_dwdr(r, h, dim, kappa):
    """Radial derivative dW/dr of Eq. 6: alpha_d h^-(d+1) (-5 q) (1 - q/2)^3, q <= kappa."""
    r = np.asarray(r, dtype=np.float64)
    q = r / h
    dw = ALPHA_WENDLAND[dim] * h ** (-dim - 1) * (-5.0 * q) * (1.0 - 0.5 * q) ** 3
    return dw if kappa is None else np.where(q <= kappa, dw, 0.0)


def lg_w(r, h, dim, kappa=KAPPA_LG):
    """Laguerre-Gauss value, Eq. 8 with the normalising constant ahat_d."""
    r = np.asarray(r, dtype=np.float64)
    q = r / h
    w = ALPHA_LG[dim] * h ** (-dim) * (1.0 - 0.5 * q * q + q ** 4 / 6.0) * np.exp(-q * q)
    return w if kappa is None else np.where(q <= kappa, w, 0.0)


def lg_dwdr(r, h, dim, kappa=KAPPA_LG):
    """dW/dr of Eq. 8: -(ahat_d h^-(d+1)) (q/3) exp(-q^2) (9 - 5 q^2 + q^4), q <= 2."""
    r = np.asarray(r, dtype=np.float64)
    q = r / h
    dw = -ALPHA_LG[dim] * h ** (-dim - 1) * (q / 3.0) * np.exp(-q * q) * (9.0 - 5.0 * q * q + q ** 4)
    return dw if kappa is None else np.where(q <= kappa, dw, 0.0)


def kernel_w(kind, r, h, dim, kappa):
    if kind == WENDLAND:
        return wendland_w(r, h, dim, kappa)
    if kind == LAGUERRE_GAUSS:
        return lg_w(r, h, dim, kappa)
    raise ValueError(kind)


def kernel_dwdr(kind, r, h, dim, kappa):
    if kind == WENDLAND:
        return wendland_dwdr(r, h, dim, kappa)
    if kind == LAGUERRE_GAUSS:
        return lg_dwdr(r, h, dim, kappa)
    raise ValueError(kind)
