"""Pins of the oracle's kernel functions (Eqs. 3, 5, 6, 8; Table 1)."""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle import kernels as K
from oracle import neighbors as N
from oracle.metrics import l2_error
from paper_2405_05155_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mass(wfun, h, dim, rmax):
    """Integral of a radial kernel over the ball r <= rmax in dim dimensions."""
    shell = {1: lambda r: 2.0, 2: lambda r: 2.0 * math.pi * r, 3: lambda r: 4.0 * math.pi * r * r}[dim]
    val, _ = integrate.quad(lambda r: shell(r) * float(wfun(r)), 0.0, rmax, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_wendland_normalisation_eq3(dim):
    # Eq. 3 with the printed alpha_d of Eq. 6 and support 2h: the integral is 1.
    h = 0.37
    m = _mass(lambda r: K.wendland_w(r, h, dim, 2.0), h, dim, 2.0 * h)
    assert abs(m - 1.0) < 1e-12


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_truncated_wendland_is_plain_cut(dim):
    # Sec. 2.3.1: truncation to 1.6h changes nothing inside 1.6h and zeroes the rest.
    h = 0.5
    r = np.linspace(0.0, 2.0 * h, 4001)
    full = K.wendland_w(r, h, dim, 2.0)
    cut = K.wendland_w(r, h, dim, 1.6)
    inside = r / h <= 1.6
    assert np.array_equal(cut[inside], full[inside])
    assert np.all(cut[~inside] == 0.0)
    # the support boundary is inclusive (Eq. 5 zeroes only |r| > kappa h)
    assert K.wendland_w(1.6 * h, h, dim, 1.6) > 0.0
    # the lost mass is small but not zero: the truncated kernel is not renormalised
    m = _mass(lambda x: K.wendland_w(x, h, dim, 1.6), h, dim, 1.6 * h)
    assert 0.985 < m < 0.9995


@pytest.mark.parametrize("kind,kappa", [(K.WENDLAND, 2.0), (K.WENDLAND, 1.6), (K.LAGUERRE_GAUSS, 2.0)])
@pytest.mark.parametrize("dim", [2, 3])
def test_derivative_matches_finite_difference(kind, kappa, dim):
    h = 0.45
    r = np.linspace(0.01, kappa * h - 0.01, 97)
    eps = 1e-6 * h
    fd = (K.kernel_w(kind, r + eps, h, dim, kappa) - K.kernel_w(kind, r - eps, h, dim, kappa)) / (2 * eps)
    an = K.kernel_dwdr(kind, r, h, dim, kappa)
    scale = np.max(np.abs(an))
    assert np.max(np.abs(fd - an)) / scale < 1e-8
    assert np.all(an < 0.0)          # monotone decreasing inside the support
    assert K.kernel_dwdr(kind, kappa * h * 1.0001, h, dim, kappa) == 0.0


@pytest.mark.parametrize("dim", [1, 2, 3])
def test_laguerre_gauss_normalisation_reading(dim):
    # Eq. 8's printed polynomial integrates to 1 over all space with ahat_d ...
    h = 1.0
    poly = lambda r: (1.0 - 0.5 * r * r + r ** 4 / 6.0) * math.exp(-r * r)
    m_inf = _mass(lambda r: K.ALPHA_LG[dim] * poly(r), h, dim, 12.0)
    assert abs(m_inf - 1.0) < 1e-12
    # ... while the printed alpha_d do not normalise it (ratio 7/5, 5/2, 7).
    ratio = K.ALPHA_LG_PRINTED[dim] / K.ALPHA_LG[dim]
    assert abs(ratio - {1: 1.4, 2: 2.5, 3: 7.0}[dim]) < 1e-12
    # cut at 2h the kernel keeps almost all of its mass; W(2)/W(0) = (5/3) e^-4
    m2 = _mass(lambda r: K.lg_w(r, h, dim), h, dim, 2.0)
    assert 0.8 < m2 < 1.0
    assert abs(K.lg_w(2.0, h, dim) / K.lg_w(0.0, h, dim) - (5.0 / 3.0) * math.exp(-4.0)) < 1e-14


def _lattice_sum_l2(kappa, h_over_dp, nx=20):
    """Eq. 10 for f = 1 with phi^n = sum_j W_ij V_j (self included) on a periodic 2D lattice."""
    dp = 1.0 / nx
    pos = inputs.lattice((nx, nx), dp)
    dom = N.Domain(2, h_over_dp * dp, kappa, (0.0, 0.0), (1.0, 1.0), (True, True))
    rp, col = N.neighbors_cells(pos, dom)
    i, j, rij, r = N.pair_geometry(pos, rp, col, dom)
    n = pos.shape[1]
    s = np.bincount(i, weights=K.wendland_w(r, dom.h, 2, kappa) * dp * dp, minlength=n)
    s = s + K.wendland_w(0.0, dom.h, 2, kappa) * dp * dp
    return l2_error(np.ones(n), s)


def test_table1_lattice_row():
    # Table 1, lattice row: 0.010 (SW, kappa = 2) and 0.006 (TW, kappa = 1.6) at h = 1.3 dp.
    with open(os.path.join(GOLDEN, "table1_lattice.json")) as f:
        g = json.load(f)
    sw = _lattice_sum_l2(2.0, g["h_over_dp"])
    tw = _lattice_sum_l2(1.6, g["h_over_dp"])
    assert round(sw, g["digits"]) == pytest.approx(g["SW_without_B"], abs=1e-12)
    assert round(tw, g["digits"]) == pytest.approx(g["TW_without_B"], abs=1e-12)
    # a renormalised truncated kernel would give a visibly different TW entry
    assert abs(tw - sw) > 0.003
