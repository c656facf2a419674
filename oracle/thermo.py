"""Canonical averages from a density of states (Eqs. 6-7 of the paper): plain float64.

TEST INFRASTRUCTURE ONLY.  u(T) = <E>/N and c(T) = (<E^2> - <E>^2) / (N T^2) with
<X> = sum_E X g(E) e^{-E/T} / sum_E g(E) e^{-E/T}, k_B = 1.
"""
from __future__ import annotations

import numpy as np


def energies(model: int, L: int) -> np.ndarray:
    N = L * L
    B = N if model == 0 else 2 * N
    k = np.arange(B + 1, dtype=np.float64)
    return -2.0 * N + (4.0 * k if model == 0 else k)


def canonical(lng, model: int, L: int, T):
    lng = np.asarray(lng, dtype=np.float64)
    E = energies(model, L)
    N = L * L
    fin = np.isfinite(lng)
    u, c = [], []
    for t in np.atleast_1d(T):
        w = lng[fin] - E[fin] / t
        w = np.exp(w - w.max())
        Z = w.sum()
        e1 = (w * E[fin]).sum() / Z
        e2c = (w * (E[fin] - e1) ** 2).sum() / Z
        u.append(e1 / N)
        c.append(e2c / (N * t * t))
    return np.array(u), np.array(c)
