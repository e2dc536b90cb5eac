"""The CUDA GELU's erf approximation (Abramowitz and Stegun 7.1.26) against its
published error bound, with the constants read from the header the kernels use."""
import math
import os
import re

import numpy as np
from scipy.special import erf

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _constants():
    text = open(os.path.join(ROOT, "paper_2405_05155_gb300", "csrc", "gelu.cuh")).read()
    found = dict(re.findall(r"\b(kP|kA[1-5])\s*=\s*(-?[0-9.]+)f", text))
    assert sorted(found) == ["kA1", "kA2", "kA3", "kA4", "kA5", "kP"]
    return {k: float(v) for k, v in found.items()}


def _erf_as(x, c):
    t = 1.0 / (1.0 + c["kP"] * x)
    poly = t * (c["kA1"] + t * (c["kA2"] + t * (c["kA3"] + t * (c["kA4"] + t * c["kA5"]))))
    return 1.0 - poly * np.exp(-x * x)


def test_erf_within_the_published_bound():
    c = _constants()
    x = np.linspace(0.0, 6.0, 200001)
    err = np.abs(_erf_as(x, c) - erf(x))
    assert err.max() <= 1.5e-7 * (1 + 1e-3)
    # float32 constants: the bound still holds to float32 resolution
    c32 = {k: float(np.float32(v)) for k, v in c.items()}
    assert np.abs(_erf_as(x, c32) - erf(x)).max() <= 2.5e-7


def test_gelu_and_derivative_forms():
    # s = (1 - erf(|z|/sqrt 2))/2, Phi(z) = 1 - s (z >= 0) or s (z < 0), and the
    # branch-free GELU(z) = max(z, 0) - |z| s the kernels use: against the erf form
    # and a central difference
    c = _constants()
    z = np.linspace(-8.0, 8.0, 4001)
    x = np.abs(z) / math.sqrt(2.0)
    s = 0.5 * (1.0 - _erf_as(x, c))
    phi = np.where(z >= 0.0, 1.0 - s, s)
    gelu = np.maximum(z, 0.0) - np.abs(z) * s
    assert np.allclose(gelu, z * phi, rtol=0, atol=1e-15)
    exact = 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))
    assert np.abs(gelu - exact).max() <= 8.0 * 1.5e-7
    grad = phi + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)
    h = 1e-5
    num = ((z + h) * 0.5 * (1 + erf((z + h) / math.sqrt(2))) - (z - h) * 0.5 * (1 + erf((z - h) / math.sqrt(2)))) / (2 * h)
    assert np.abs(grad - num).max() < 1e-6
