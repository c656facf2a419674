"""Seeded synthetic inputs shared by the oracle-side and the CUDA-side tests.

Holds no arithmetic of the method: only numpy draws of lattices, ln g arrays,
histograms and random words with the shapes of the REWL workloads.
"""
import numpy as np

WORKLOADS = {
    # name: (model, L, windows, walkers per window, ln f final)
    "ising_L8_h4_m1": (0, 8, 4, 1, 1e-6),
    "ising_L64_h32_m16": (0, 64, 32, 16, 1e-8),
    "potts10_L40_h64_m16": (10, 40, 64, 16, 1e-8),
}


def seed_for(config_id: int, instance: int = 0) -> int:
    return 0x5EED201400000000 + config_id * 1000 + instance


def random_lattices(rng, model, L, n):
    if model == 0:
        return (rng.integers(0, 2, size=(n, L * L)) * 2 - 1).astype(np.int8)
    return rng.integers(0, model, size=(n, L * L)).astype(np.int8)


def random_words(rng, n, cols=3):
    return rng.integers(0, 2 ** 32, size=(n, cols), dtype=np.uint64).astype(np.uint32)


def random_lng(rng, n, W, scale=3.0, offset=0.0):
    """Smooth-ish random ln g rows (a random walk) so that accept ratios vary."""
    steps = rng.normal(0.0, scale, size=(n, W))
    return (np.cumsum(steps, axis=1) + offset).astype(np.float64)


def random_H(rng, n, W, hi=1000):
    return rng.integers(0, hi, size=(n, W)).astype(np.uint32)
