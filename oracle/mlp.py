"""Learned relaxation proposal, oracle version (test infrastructure).

The paper has no learned component; this restates the network the benchmark
configuration asks for, in float64, so that the GPU's bfloat16 tensor-core
forward and backward passes have a reference:

* features of particle i (97 used, padded to 128): the offsets (x_j - x_i)/h of
  its 32 nearest neighbours within the Laguerre-Gauss support (cut-off 2h),
  ordered by (squared distance, j), zero-filled when fewer than 32 exist, then
  phi_i / h (the signed distance to the body surface);
* network: 128 -> 128 -> 128 -> 128 -> 3 with GELU (erf form) after each of the
  three hidden layers; output = predicted displacement / h;
* parameters (flat float layout shared with the GPU): W1 (128x128, out x in), b1,
  W2, b2, W3, b3, W4 (3x128), b4;
* loss: mean squared error over the batch and the 3 outputs;
* optimiser: Adam (beta1 = 0.9, beta2 = 0.999, eps = 1e-8) with bias correction.
"""
import math

import numpy as np
from scipy.special import erf

from .neighbors import pair_geometry, squared_distance

N_NEIGH = 32
N_IN = 128
N_HID = 128
N_OUT = 3
SHAPES = [("W1", (N_HID, N_IN)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_OUT, N_HID)), ("b4", (N_OUT,))]
N_PARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def unflatten(flat):
    out = {}
    o = 0
    for name, shape in SHAPES:
        k = int(np.prod(shape))
        out[name] = np.asarray(flat[o:o + k], dtype=np.float64).reshape(shape)
        o += k
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel() for name, _ in SHAPES])


def features(pos, row_ptr, col, dom, phi):
    """(n, 128) float64 features from the neighbour lists (any cut-off >= the nearest 32)."""
    n = pos.shape[1]
    i, j, rij, r = pair_geometry(pos, row_ptr, col, dom)
    d2 = squared_distance(rij)
    order = np.lexsort((j, d2, i))              # by row, then squared distance, then index
    i, j, d2 = i[order], j[order], d2[order]
    rij = rij[:, order]
    start = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(i, minlength=n), out=start[1:])
    rank = np.arange(i.size) - start[i]
    keep = rank < N_NEIGH
    X = np.zeros((n, N_IN))
    for a in range(3):
        # offsets x_j - x_i = -r_ij
        X[i[keep], 3 * rank[keep] + a] = -rij[a, keep] / dom.h
    X[:, 3 * N_NEIGH] = phi / dom.h
    return X


def gelu(z):
    return 0.5 * z * (1.0 + erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(flat, X):
    p = unflatten(flat)
    cache = {"X": X}
    h = X
    for l in (1, 2, 3):
        z = h @ p["W%d" % l].T + p["b%d" % l]
        cache["Z%d" % l] = z
        h = gelu(z)
        cache["H%d" % l] = h
    y = h @ p["W4"].T + p["b4"]
    return y, cache


def loss_and_grad(flat, X, T):
    """MSE loss and its gradient with respect to the flat parameters (manual backprop)."""
    p = unflatten(flat)
    y, c = forward(flat, X)
    B = X.shape[0]
    diff = y - T
    loss = float(np.sum(diff * diff) / (B * N_OUT))
    dY = 2.0 * diff / (B * N_OUT)
    g = {"W4": dY.T @ c["H3"], "b4": dY.sum(axis=0)}
    dH = dY @ p["W4"]
    for l in (3, 2, 1):
        dZ = dH * gelu_grad(c["Z%d" % l])
        below = c["H%d" % (l - 1)] if l > 1 else c["X"]
        g["W%d" % l] = dZ.T @ below
        g["b%d" % l] = dZ.sum(axis=0)
        dH = dZ @ p["W%d" % l]
    return loss, flatten(g)


def adam(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; ``step`` counts from 1."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return flat - lr * mhat / (np.sqrt(vhat) + eps), m, v
