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


def smooth_concave_lng(B, peak, top, low=0.7):
    """A synthetic ln g over bins 0..B with the shape of a lattice density of states: `low` at
    bin 0, rising to `top` at bin `peak`, falling back to half of `top` at bin B."""
    k = np.arange(B + 1, dtype=np.float64)
    up = low + (top - low) * (1.0 - (1.0 - k / peak) ** 2)
    down = top - 0.5 * top * ((k - peak) / max(B - peak, 1)) ** 2
    return np.where(k <= peak, up, down)


def late_stage_state(rng, lo, hi, W, m, lng_bins, valid, step, lnf_final):
    """A state deep into a run, for planting on both sides: every walker's ln g is
    lng_bins over its window plus small per-walker noise (0 on bins never visited), H near
    flat (one walker of every fourth window has a short bin), and windows cycle through four
    kinds: halving mode at ln f = 2^-26 (all flat / one short bin), 1/t mode at the
    non-dyadic ln f = visited bins / moves, and finished (frozen, 1/t mode, ln f below
    ln f_final).  Every slot has made `step` moves."""
    h = len(lo)
    nw = h * m
    out = dict(lng=np.zeros((nw, W)), H=np.zeros((nw, W), np.uint32),
               mask=np.zeros((h, W), np.uint8), lnf=np.zeros(h), mode=np.zeros(h, np.uint8),
               iter=np.zeros(h, np.int32), finished=np.zeros(h, np.uint8),
               flat=np.zeros(nw, np.uint8), step=np.full(nw, step, np.uint64))
    for w in range(h):
        nb = int(hi[w] - lo[w] + 1)
        v = np.asarray(valid[lo[w]:hi[w] + 1], bool)
        out["mask"][w, :nb] = v
        kind = w % 4
        for i in range(m):
            g = w * m + i
            out["lng"][g, :nb] = np.where(v, lng_bins[lo[w]:hi[w] + 1] + rng.normal(0, 1e-3, nb), 0.0)
            Hr = rng.integers(45_000, 55_000, nb)
            if kind == 1 and i == m - 1:
                Hr[nb // 2] = 1000
            out["H"][g, :nb] = np.where(v, Hr, 0)
        if kind in (0, 1):
            out["lnf"][w], out["iter"][w] = 2.0 ** -26, 26
        elif kind == 2:
            out["lnf"][w], out["mode"][w], out["iter"][w] = float(v.sum()) / float(step), 1, 31
        else:
            out["lnf"][w], out["mode"][w], out["iter"][w] = 0.7 * lnf_final, 1, 33
            out["finished"][w] = 1
    return out
