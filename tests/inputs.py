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


def mlp_params(seed, nparam=4481, scale=0.3):
    """Random MLP parameter vector (float32-representable) for the gradient tests."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, scale, nparam).astype(np.float32).astype(np.float64)


def mlp_data(seed, n):
    """Features (e in [-2, 0], q in {2, 10}, 1/L in [1/32, 1/8]) and smooth targets."""
    rng = np.random.default_rng(seed)
    e = rng.uniform(-2.0, 0.0, n)
    q = rng.choice([2.0, 10.0], n)
    il = 1.0 / rng.choice([8.0, 12.0, 16.0, 24.0, 32.0], n)
    X = np.stack([e, q, il], axis=1).astype(np.float32)
    T = (np.log(q) * (1 + e / 2.0) ** 0.5 * (1 - il)).astype(np.float32)
    return X, T
