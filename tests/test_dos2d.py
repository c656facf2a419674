"""Joint density of states g(E, M) (Sec. 3, Eqs. 3-4): pins of the oracle.

* exact g(E, M): enumeration = transfer matrix (4x4); marginals over M equal the exact g(E)
  (5x5, the 6x6 golden file); M -> -M symmetry; sum = 2^N;
* the deterministic logarithm used for fragments against libm;
* the measurement counts each walker's (bin, up spins) once per round (recounted here from
  the lattices);
* fragments by hand; joining exact fragments with arbitrary window offsets returns the exact
  surface; the join picks the point where the normals coincide and Eq. (4) averages g;
* a production run after convergence gives g(E, M) of the 4x4 lattice within its error.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from oracle import exact_dos as X

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
EX4 = X.brute_force_ising_em(4)


def load_em(name, N):
    g = np.zeros((N + 1, N + 1), dtype=object)
    for line in open(os.path.join(GOLDEN, name)):
        if line.startswith("#"):
            continue
        k, j, v = line.split()
        g[int(k), int(j)] = int(v)
    return g


def ln_exact(g):
    return np.array([[math.log(int(v)) if v else -math.inf for v in row] for row in g])


def test_exact_em_enumeration_and_transfer_matrix():
    b4 = X.brute_force_ising_em(4)
    assert np.array_equal(b4, X.transfer_matrix_ising_em(4))
    assert b4.sum() == 2 ** 16 and np.array_equal(b4, b4[:, ::-1])
    assert b4[0, 0] == 1 and b4[0, 16] == 1 and b4[0, 1:16].sum() == 0
    # one flipped spin: 4 unsatisfied bonds (k = 2), M = +-(N-2)
    assert b4[2, 1] == 16 and b4[2, 15] == 16
    assert [int(v) for v in b4.sum(axis=1)] == X.brute_force_ising(4)
    t5 = X.transfer_matrix_ising_em(5)
    assert [int(v) for v in t5.sum(axis=1)] == X.transfer_matrix_ising(5)
    assert t5.sum() == 2 ** 25 and np.array_equal(t5, t5[:, ::-1])


def test_golden_6x6_em():
    g = load_em("ising_L6_em_counts.txt", 36)
    assert sum(int(v) for v in g.ravel()) == 2 ** 36
    assert [sum(int(v) for v in row) for row in g] == X.transfer_matrix_ising(6)
    assert all(g[k, j] == g[k, 36 - j] for k in range(37) for j in range(37))


def test_deterministic_log():
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.integers(1, 2 ** 62, 20000).astype(np.float64),
                         rng.uniform(0.5, 4.0, 20000), 2.0 ** np.arange(-30, 60)])
    for x in xs:
        a, b = O.ln(x), math.log(x)
        assert abs(a - b) <= 4 * math.ulp(b) + 1e-300, (x, a, b)
    assert O.ln(1.0) == 0.0


def test_measurement_counts_each_walker_once_per_round():
    r = O.REWL(0, 4, 3, 0.75, 2, 1e-2, 0.8, seed=21, interval=50)
    assert r.init() == 0
    r.measure_em(True)
    prev = r.hist_em().astype(np.int64)
    for _ in range(12):
        r.round()
        cur = r.hist_em().astype(np.int64)
        inc = cur - prev
        prev = cur
        assert inc.sum() == r.h * r.m
        # counted points lie in their windows and are reachable (E, M) points
        for w in range(r.h):
            for b, j in zip(*np.nonzero(inc[w])):
                assert 0 <= b <= r.hi[w] - r.lo[w]
                assert EX4[r.lo[w] + b, j] > 0
    with pytest.raises(ValueError):
        O.REWL(3, 4, 2, 0.75, 1, 1e-2, 0.8, seed=1).measure_em(True)


def test_measurement_recount_without_exchange():
    """h = 1: no exchange, so the lattices after a round are the measured ones."""
    r = O.REWL(0, 4, 1, 0.75, 3, 1e-2, 0.8, seed=5, interval=37)
    assert r.init() == 0
    r.measure_em(True)
    expect = np.zeros((1, r.W, 17), np.int64)
    for _ in range(20):
        r.round()
        st = r.state()
        for g in range(3):
            expect[0, st["k"][g] - r.lo[0], int((st["spins"][g] > 0).sum())] += 1
    assert np.array_equal(r.hist_em().astype(np.int64), expect)


def test_fragments_by_hand():
    lo, hi = np.array([0, 2]), np.array([3, 4])
    W, N1 = 4, 4
    mean = np.array([[0.5, 1.0, 2.0, 3.0], [10.0, 11.0, 12.0, 0.0]])
    valid = np.array([[1, 1, 0, 1], [1, 1, 1, 0]], np.uint8)
    hem = np.zeros((2, W, N1), np.uint32)
    hem[0, 0] = [0, 2, 6, 0]
    hem[0, 2] = [1, 1, 1, 1]   # unvisited bin: absent whatever the counts
    hem[1, 1] = [5, 0, 0, 0]
    S = O.frag_em(lo, hi, mean, valid, hem)
    assert S[0, 0, 1] == pytest.approx(0.5 + math.log(2 / 8), abs=1e-15)
    assert S[0, 0, 2] == pytest.approx(0.5 + math.log(6 / 8), abs=1e-15)
    assert np.isneginf(S[0, 0, 0]) and np.isneginf(S[0, 0, 3])
    assert np.all(np.isneginf(S[0, 2])) and np.all(np.isneginf(S[0, 1]))
    assert S[1, 1, 0] == 11.0 and np.all(np.isneginf(S[1, 1, 1:]))


def _cut(lex, lo, hi, W, offsets):
    h = len(lo)
    S = np.full((h, W, lex.shape[1]), -np.inf)
    for w in range(h):
        S[w, : hi[w] - lo[w] + 1] = lex[lo[w]: hi[w] + 1] + offsets[w]
    return S


def test_join_exact_fragments_returns_exact_surface():
    N = 36
    lex = ln_exact(load_em("ising_L6_em_counts.txt", N))
    B = N
    for h in (2, 4, 6):
        lo, hi = O.windows(B, h, 0.75)
        W = int((hi - lo).max()) + 1
        offs = np.random.default_rng(h).normal(0, 50, h)
        out, joins = O.join_em(lo, hi, _cut(lex, lo, hi, W, offs), B, N)
        fin = np.isfinite(lex)
        assert np.array_equal(np.isfinite(out), fin)
        ref = lex - (np.log(np.exp(lex[fin] - lex[fin].max()).sum()) + lex[fin].max()) + N * math.log(2)
        assert np.max(np.abs(out[fin] - ref[fin])) < 1e-11
        for w, (k, j) in enumerate(joins):
            assert lo[w + 1] <= k <= hi[w] and fin[k, j]


def test_join_picks_point_where_normals_agree_and_averages():
    """Two fragments whose surfaces differ by c + eps * ((k-k0)^2 + (j-j0)^2): the normals
    agree only at (k0, j0) (the stencils are exact for quadratics), so the join is there,
    window 1 is shifted by -c, and Eq. (4) averages g where both are present."""
    B, N = 30, 20
    lo, hi = np.array([0, 12]), np.array([20, 30])
    W, N1 = 21, N + 1
    kk, jj = np.meshgrid(np.arange(B + 1), np.arange(N1), indexing="ij")
    base = 0.02 * (kk - 15.0) ** 2 - 0.03 * (jj - 10.0) ** 2 + 0.1 * kk * jj / 10
    k0, j0, c, eps = 16, 7, 5.0, 0.01
    other = base + c + eps * ((kk - k0) ** 2 + (jj - j0) ** 2)
    S = np.full((2, W, N1), -np.inf)
    S[0, :21] = base[0:21]
    S[1, :19] = other[12:31]
    out, joins = O.join_em(lo, hi, S, B, N)
    assert tuple(joins[0]) == (k0, j0)
    # undo the normalisation with a point only window 0 covers
    shift0 = out[3, 4] - base[3, 4]
    a, b = base[18, 9], other[18, 9] - c
    assert out[18, 9] - shift0 == pytest.approx(math.log((math.exp(a) + math.exp(b)) / 2), abs=1e-12)
    assert out[25, 3] - shift0 == pytest.approx(other[25, 3] - c, abs=1e-12)


def test_join_normals_in_physical_units():
    """Normals use dE = 4 per bin and dM = 2 per up spin.  Only two points have normals in
    both fragments (plus-shaped patches): window 1 has gradient (2, 0) per index at P1 and
    (0, 1.5) at P2, window 0 is flat.  In physical units |grad|^2 is 0.25 at P1 and 0.5625 at
    P2, so the join is at P1 (in index units it would be P2)."""
    B, N = 30, 20
    lo, hi = np.array([0, 10]), np.array([20, 30])
    W, N1 = 21, N + 1
    A = np.full((B + 1, N1), -np.inf)
    Bf = np.full((B + 1, N1), -np.inf)
    P1, P2 = (14, 5), (17, 12)
    for (k, j) in (P1, P2):
        for (dk, dj) in ((0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)):
            A[k + dk, j + dj] = 0.0
            Bf[k + dk, j + dj] = 0.0
    Bf[15, 5], Bf[13, 5] = 2.0, -2.0
    Bf[17, 13], Bf[17, 11] = 1.5, -1.5
    S = np.full((2, W, N1), -np.inf)
    S[0, :21] = A[0:21]
    S[1, :21] = Bf[10:31]
    _, joins = O.join_em(lo, hi, S, B, N)
    assert tuple(joins[0]) == P1


def test_join_ties_take_smallest_point():
    """Two flat fragments: every candidate's normals coincide exactly; the join is the first
    point (smallest bin, then smallest j) where both fragments have a normal."""
    B, N = 30, 20
    lo, hi = np.array([0, 10]), np.array([20, 30])
    S = np.full((2, 21, N + 1), -np.inf)
    S[0, :21] = 0.0
    S[1, :21] = 3.0
    out, joins = O.join_em(lo, hi, S, B, N)
    assert tuple(joins[0]) == (11, 1)
    assert np.all(out == out[0, 0])  # one flat surface after the shift


def test_production_run_gives_exact_g_em_4x4():
    ex = EX4
    lex = np.where(ex > 0, np.log(np.maximum(ex, 1)), -np.inf)
    fin = np.isfinite(lex)
    errs = []
    for seed in range(3):
        r = O.REWL(0, 4, 3, 0.75, 2, 1e-6, 0.8, seed=40 + seed, interval=100)
        assert r.init() == 0
        r.run(10 ** 7)
        r.measure_em(True)
        r.set_production(True)
        assert r.run(3000) == 3000
        out, joins = r.stitch_em()
        assert np.array_equal(np.isfinite(out), fin)
        errs.append(np.abs(out[fin] - lex[fin]))
    errs = np.array(errs)
    assert errs.max() < 0.6, errs.max()
    assert errs.mean() < 0.12, errs.mean()
