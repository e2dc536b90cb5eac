"""Pins of the oracle's learned-proposal network (features, GELU, backprop, Adam)."""
import math

import numpy as np
import pytest

from oracle import mlp as OM
from oracle import neighbors as ON
from paper_2405_05155_gb300 import inputs


def test_gelu_definition_and_derivative():
    z = np.linspace(-6, 6, 1001)
    # erf form: 0.5 z (1 + erf(z / sqrt 2)) = z Phi(z); Phi by quadrature-free identities
    assert abs(OM.gelu(np.array([0.0]))[0]) == 0.0
    assert abs(OM.gelu(np.array([1.0]))[0] - 0.8413447460685429) < 1e-15
    assert abs(OM.gelu(np.array([-1.0]))[0] + 0.15865525393145707) < 1e-15
    eps = 1e-6
    fd = (OM.gelu(z + eps) - OM.gelu(z - eps)) / (2 * eps)
    assert np.max(np.abs(fd - OM.gelu_grad(z))) < 1e-8


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    flat = inputs.mlp_init(3)
    X = rng.normal(size=(6, OM.N_IN))
    T = rng.normal(size=(6, OM.N_OUT))
    loss, g = OM.loss_and_grad(flat, X, T)
    idx = rng.choice(OM.N_PARAM, 60, replace=False)
    # every parameter block is probed
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in OM.SHAPES])
    idx = np.concatenate([idx, offs[:-1], offs[1:] - 1])
    eps = 1e-6
    for k in idx:
        fp = flat.copy()
        fp[k] += eps
        fm = flat.copy()
        fm[k] -= eps
        fd = (OM.loss_and_grad(fp, X, T)[0] - OM.loss_and_grad(fm, X, T)[0]) / (2 * eps)
        assert abs(fd - g[k]) <= 1e-6 * max(1e-3, abs(g[k])) + 1e-10, (k, fd, g[k])


def test_adam_matches_hand_computation():
    w = np.array([1.0, -2.0])
    g = np.array([0.5, -0.25])
    m = np.zeros(2)
    v = np.zeros(2)
    w1, m1, v1 = OM.adam(w, g, m, v, 1, 1e-3)
    # first step: mhat = g, vhat = g^2, so w -= lr g / (|g| + eps)
    assert np.allclose(w1, w - 1e-3 * g / (np.abs(g) + 1e-8), atol=1e-15)
    w2, m2, v2 = OM.adam(w1, g, m1, v1, 2, 1e-3)
    mh = (0.9 * 0.1 * g + 0.1 * g) / (1 - 0.81)
    vh = (0.999 * 0.001 * g * g + 0.001 * g * g) / (1 - 0.999 ** 2)
    assert np.allclose(w2, w1 - 1e-3 * mh / (np.sqrt(vh) + 1e-8), atol=1e-15)


def test_features_on_a_lattice():
    # simple cubic lattice: the 6 nearest neighbours sit at distance dp along the axes
    dp = 0.1
    pos = inputs.lattice((8, 8, 8), dp)
    dom = ON.Domain(3, 1.3 * dp, 2.0, [0.0] * 3, [0.8] * 3, [True] * 3)
    rp, col = ON.neighbors_cells(pos, dom)
    phi = np.full(pos.shape[1], -0.3)
    X = OM.features(pos, rp, col, dom, phi)
    i = 0
    first6 = X[i, :18].reshape(6, 3) * dom.h
    assert np.allclose(np.sort(np.linalg.norm(first6, axis=1)), dp, atol=1e-12)
    # ties in distance are broken by ascending j
    js = col[rp[i]:rp[i + 1]]
    dx = ON.min_image(pos[:, js] - pos[:, [i]], dom)
    d2 = ON.squared_distance(dx)
    best = js[np.lexsort((js, d2))][:6]
    expect = ON.min_image(pos[:, best] - pos[:, [i]], dom).T
    assert np.allclose(first6, expect, atol=1e-12)
    assert np.all(X[:, 96] == -0.3 / dom.h)
    assert np.all(X[:, 97:] == 0.0)
    # 80 neighbours at 2h = 2.6 dp: all 32 slots are filled
    assert np.all(np.linalg.norm(X[:, 93:96], axis=1) > 0)
