"""Float64 reference of the warm-start MLP (3 -> 64 -> 64 -> 1, tanh, mean squared error).

TEST INFRASTRUCTURE ONLY: the tests compare the CUDA training kernels' forward pass,
gradients and Adam steps with these functions, and pin these functions by central
differences.  The CUDA library never imports this module.

Parameter vector layout (shared only as a documented convention, not as code):
W1[64][3], b1[64], W2[64][64] (W2[i][j]: from hidden-1 unit j to hidden-2 unit i), b2[64],
W3[64], b3 — 4481 numbers.
Features of one energy bin (Potts convention for both models): e = E/N with Ising mapped by
E_P = (E_I - 2N)/2, then q and 1/L; target ln g(E)/N (g normalised to sum q^N).
"""
from __future__ import annotations

import numpy as np

H = 64
NPARAM = H * 3 + H + H * H + H + H + 1


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * 3].reshape(H, 3); o += H * 3
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def forward(p, X):
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    h1 = np.tanh(X @ W1.T + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3 + b3, (h1, h2)


def loss_and_grad(p, X, T):
    """Mean squared error and its gradient by back-propagation (chain rule, layer by layer)."""
    W1, b1, W2, b2, W3, b3 = unpack(p)
    X = np.asarray(X, dtype=np.float64)
    T = np.asarray(T, dtype=np.float64)
    y, (h1, h2) = forward(p, X)
    n = len(T)
    r = y - T
    loss = float(np.mean(r * r))
    dy = 2.0 * r / n
    gW3 = h2.T @ dy
    gb3 = dy.sum()
    dz2 = np.outer(dy, W3) * (1.0 - h2 * h2)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * (1.0 - h1 * h1)
    gW1 = dz1.T @ X
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g


def adam(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (Kingma & Ba 2015); t counts from 1."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def features(model: int, L: int, ks):
    """(e, q, 1/L) of bins ks; e in the Potts convention."""
    N = L * L
    ks = np.asarray(ks, dtype=np.float64)
    q = 2 if model == 0 else model
    e = (-2.0 + 2.0 * ks / N) if model == 0 else (-2.0 + ks / N)
    return np.stack([e, np.full_like(e, q), np.full_like(e, 1.0 / L)], axis=1)


def init_params(seed: int = 0):
    """Glorot-uniform weights, zero biases."""
    rng = np.random.default_rng(seed)
    def glorot(o, i):
        a = np.sqrt(6.0 / (i + o))
        return rng.uniform(-a, a, size=(o, i))
    return np.concatenate([glorot(H, 3).ravel(), np.zeros(H), glorot(H, H).ravel(),
                           np.zeros(H), glorot(1, H).ravel(), [0.0]])
