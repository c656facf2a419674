"""Joint density of states g(E, M) on the GPU (Sec. 3, Eqs. 3-4) against the oracle.

The (E, M) histogram and the production rounds are integer/bit-exact; the join points are
identical (the normals are computed with the same float64 operations in the same order);
joined values agree to round-off (exp / log1p / the normalising sum differ in the last bits).
"""
import math
import os

import numpy as np
import pytest

import oracle as O

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
FIELDS = ["spins", "k", "lng", "H", "step", "acc", "flat", "lnf", "iter", "finished", "mask",
          "swap_att", "swap_acc", "round"]


@pytest.fixture(scope="module")
def R():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1402_2328_gb300 import build as B
    B.build()
    import paper_1402_2328_gb300.rewl as R
    return R


def _same(a, b):
    for f in FIELDS:
        x, y = np.asarray(a[f]), np.asarray(b[f])
        if x.dtype.kind == "f":
            assert np.array_equal(x.view(np.uint64), y.view(np.uint64)), f
        else:
            assert np.array_equal(x, y), f


def _close(a, b, tol=1e-11):
    fa, fb = np.isfinite(a), np.isfinite(b)
    assert np.array_equal(fa, fb)
    assert np.max(np.abs(a[fa] - b[fa])) <= tol * max(1.0, np.max(np.abs(b[fb])))


def load_em(name, N):
    g = np.full((N + 1, N + 1), -np.inf)
    for line in open(os.path.join(GOLDEN, name)):
        if not line.startswith("#"):
            k, j, v = line.split()
            g[int(k), int(j)] = math.log(int(v))
    return g


def _pair(L, h, m, lnf_final, seed, interval):
    import paper_1402_2328_gb300.rewl as R
    g = R.REWL(0, L, h, 0.75, m, lnf_final, 0.8, seed=seed, interval=interval)
    o = O.REWL(0, L, h, 0.75, m, lnf_final, 0.8, seed=seed, interval=interval)
    g.init()
    assert o.init() == 0
    return g, o


def test_measurement_and_production_bit_exact(R):
    g, o = _pair(6, 3, 2, 1e-3, seed=71, interval=300)
    g.run(max_rounds=15)
    o.run(15)
    g.set_param("measure_em", 1)
    o.measure_em(True)
    g.run(max_rounds=25)
    o.run(25)
    assert np.array_equal(g.hist_em(), o.hist_em())
    _same(g.state(), o.state())
    assert g.run() == "done"
    o.run(10 ** 6)
    _same(g.state(), o.state())
    # production: frozen ln g, rounds go on until the budget
    g.set_param("production", 1)
    o.set_production(True)
    lng0 = g.get_state("lng").copy()
    assert g.run(max_rounds=60) == "budget"
    assert o.run(60) == 60
    st = g.state()
    assert np.array_equal(st["lng"], lng0) and st["round"] == o.state()["round"]
    assert np.array_equal(g.hist_em(), o.hist_em())
    _same(st, o.state())
    a, ja = g.stitch_em()
    b, jb = o.stitch_em()
    assert np.array_equal(ja, jb)
    _close(a, b)
    g.set_param("production", 0)
    assert g.run(max_rounds=5) == "done"
    g.close()


def test_join_em_synthetic_fragments(R):
    """Exact 6x6 g(E, M) cut into windows with offsets and noise, points removed: the GPU
    join equals the oracle's; without noise it returns the exact surface."""
    N, B = 36, 36
    lex = load_em("ising_L6_em_counts.txt", N)
    rng = np.random.default_rng(5)
    for h, noise, drop in [(3, 0.0, 0.0), (4, 0.05, 0.1), (6, 0.2, 0.3)]:
        lo, hi = O.windows(B, h, 0.75)
        W = int((hi - lo).max()) + 1
        S = np.full((h, W, N + 1), -np.inf)
        for w in range(h):
            blk = lex[lo[w]: hi[w] + 1] + rng.normal(0, 30) + rng.normal(0, noise, (hi[w] - lo[w] + 1, N + 1))
            blk[rng.random(blk.shape) < drop] = -np.inf
            S[w, : hi[w] - lo[w] + 1] = blk
        ref, jref = O.join_em(lo, hi, S, B, N)
        St = torch.from_numpy(S).cuda()
        out = torch.zeros((B + 1, N + 1), dtype=torch.float64, device="cuda")
        joins = R.join_em(St, lo, hi, B, out)
        torch.cuda.synchronize()
        assert np.array_equal(joins, jref), (h, joins, jref)
        _close(out.cpu().numpy(), ref)
        if noise == 0.0:
            fin = np.isfinite(lex)
            norm = lex - (np.log(np.exp(lex[fin] - lex[fin].max()).sum()) + lex[fin].max()) + N * math.log(2)
            assert np.max(np.abs(out.cpu().numpy()[fin] - norm[fin])) < 1e-10


def test_join_em_many_blocks(R):
    """A smooth random surface on a large grid (several blocks per pair, ragged tail)."""
    B, N1, h = 300, 257, 9
    lo, hi = O.windows(B, h, 0.75)
    W = int((hi - lo).max()) + 1
    kk, jj = np.meshgrid(np.arange(B + 1) / B, np.arange(N1) / N1, indexing="ij")
    base = 40 * np.sin(2.1 * kk + 0.3) * np.cos(1.3 * jj - 0.2) + 9 * kk * jj
    rng = np.random.default_rng(9)
    S = np.full((h, W, N1), -np.inf)
    for w in range(h):
        blk = base[lo[w]: hi[w] + 1] + rng.normal(0, 10) + rng.normal(0, 1e-3, (hi[w] - lo[w] + 1, N1))
        S[w, : hi[w] - lo[w] + 1] = blk
    ref, jref = O.join_em(lo, hi, S, B, N1 - 1)
    out = torch.zeros((B + 1, N1), dtype=torch.float64, device="cuda")
    joins = R.join_em(torch.from_numpy(S).cuda(), lo, hi, B, out)
    torch.cuda.synchronize()
    assert np.array_equal(joins, jref)
    _close(out.cpu().numpy(), ref)


def test_production_gives_g_em_6x6(R):
    """Converged REWL, then production rounds with the (E, M) measurement: the joined
    g(E, M) of the 6x6 lattice against the exact one (transfer matrix)."""
    lex = load_em("ising_L6_em_counts.txt", 36)
    fin = np.isfinite(lex)
    r = R.REWL(0, 6, 4, 0.75, 4, 1e-6, 0.8, seed=404, interval=1000)
    assert r.run() == "done"
    r.set_param("measure_em", 1)
    r.set_param("production", 1)
    r.run(max_rounds=3000)
    out, joins = r.stitch_em()
    fo = np.isfinite(out)
    assert np.all(fo <= fin)                      # never a point that does not exist
    assert fo.sum() >= 0.9 * fin.sum()
    # weight the error by how likely the point is at its energy
    ex = np.where(fin, np.exp(lex - lex.max()), 0)
    rs = ex.sum(axis=1, keepdims=True)
    pm = np.divide(ex, rs, out=np.zeros_like(ex), where=rs > 0)
    sel = fo & (pm > 1e-2)
    d = np.abs(out[sel] - lex[sel])
    assert d.max() < 0.6 and d.mean() < 0.15, (d.max(), d.mean())
    r.close()


def test_em_errors(R):
    p = R.REWL(10, 8, 2, 0.75, 1, 1e-3, 0.8, seed=1)
    with pytest.raises(R.REWLError):
        p.set_param("measure_em", 1)
    p.close()
    g = R.REWL(0, 8, 2, 0.75, 1, 1e-3, 0.8, seed=1)
    g.init()
    with pytest.raises(R.REWLError):
        g.hist_em()
    g.close()
