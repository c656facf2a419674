"""Whole-run pins of the REWL oracle (Sec. 2, Eq. 1; Sec. 3, Eq. 2).

* prep leaves every walker inside its window with a consistent bin;
* the ln f schedule halves until below ln f_final;
* converged runs reproduce exact g(E) (enumeration / Kaufman) within the
  statistical error, with and without replica exchange, for Ising and Potts;
* detailed balance of moves + exchanges with nearly frozen, window-specific ln g:
  the visit histograms follow exp(-tilt) exactly as the exchange rule requires;
* joining reproduces an exact g(E) cut into shifted windows to round-off, and picks
  the bin where the derivatives agree.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact_dos as X


def _exact(model, L, q=2):
    ex = np.array(X.exact_lng(model, L, q))
    return X.normalise_lng(ex, L * L * math.log(q))


def test_prep_puts_walkers_in_windows():
    for model, L, h in [(0, 16, 8), (10, 12, 8), (3, 8, 4)]:
        r = O.REWL(model, L, h, 0.75, 3, 1e-3, 0.8, seed=42 + model, interval=100)
        assert r.init() == 0
        st = r.state()
        N = L * L
        for g in range(h * 3):
            w = g // 3
            E = O.energy(model, L, st["spins"][g])
            kb = (E + 2 * N) // (4 if model == 0 else 1)
            assert st["k"][g] == kb and r.lo[w] <= kb <= r.hi[w]
        assert np.all(st["step"] == 0)


def test_lnf_schedule_halving():
    r = O.REWL(0, 4, 2, 0.75, 2, 1e-6, 0.8, seed=5, interval=500)
    assert r.init() == 0
    r.run(10 ** 6)
    st = r.state()
    # ln f = 2^0 ... 2^-19 are run (>= 1e-6); 2^-20 < 1e-6 ends the window
    assert np.all(st["finished"] == 1)
    assert np.all(st["iter"] == 20) and np.all(st["lnf"] == 2.0 ** -20)
    # a finished window keeps its walkers identical (averaged, then frozen)
    lng = st["lng"].reshape(2, 2, -1)
    assert np.array_equal(lng[:, 0], lng[:, 1])


@pytest.mark.parametrize("model,L,q,h,m,tol", [(0, 4, 2, 1, 8, 0.12), (0, 4, 2, 3, 6, 0.12),
                                              (3, 3, 3, 2, 6, 0.25), (2, 4, 2, 2, 6, 0.12)])
def test_converges_to_exact(model, L, q, h, m, tol):
    ex = _exact(model, L, q)
    fin = np.isfinite(ex)
    errs, bias = [], np.zeros(len(ex))
    for seed in range(4):
        r = O.REWL(model, L, h, 0.75, m, 1e-6, 0.8, seed=1000 + seed, interval=200)
        assert r.init() == 0
        r.run(10 ** 7)
        out, _ = r.stitch(0)
        assert np.array_equal(np.isfinite(out), fin)
        d = np.where(fin, out - np.where(fin, ex, 0), 0)
        errs.append(np.abs(d).max())
        bias += d / 4
    assert max(errs) < tol, errs
    assert np.abs(bias).max() < tol / 2, bias


def test_caller_windows():
    """Windows given by the caller: the equal layout passed explicitly reproduces the default
    run bit for bit, and an uneven layout (Fig. 1b style) still converges to the exact g(E)."""
    a = O.REWL(0, 6, 3, 0.75, 2, 1e-3, 0.8, seed=77, interval=300)
    b = O.REWL(0, 6, 3, 0.75, 2, 1e-3, 0.8, seed=77, interval=300, lo_hi=O.windows(36, 3, 0.75))
    for r in (a, b):
        assert r.init() == 0
        r.run(25)
    sa, sb = a.state(), b.state()
    for f in ("spins", "k", "lng", "H", "lnf", "swap_acc"):
        assert np.array_equal(np.asarray(sa[f]), np.asarray(sb[f])), f
    with pytest.raises(ValueError):
        O.REWL(0, 4, 2, 0.75, 1, 1e-3, 0.8, seed=1, lo_hi=([0, 9], [8, 16]))  # no overlap
    ex = _exact(0, 4)
    fin = np.isfinite(ex)
    errs = []
    for seed in range(3):
        r = O.REWL(0, 4, 3, 0.75, 4, 1e-6, 0.8, seed=300 + seed, interval=200,
                   lo_hi=([0, 3, 6], [6, 10, 16]))
        assert r.init() == 0
        r.run(10 ** 7)
        out, _ = r.stitch(0)
        assert np.array_equal(np.isfinite(out), fin)
        errs.append(np.abs(out[fin] - ex[fin]).max())
    assert max(errs) < 0.12, errs


def test_prep_reaches_narrow_top_windows():
    """Narrow windows at the top of the Ising range: the greedy walk from a random lattice
    stalls below them; the restart from the checkerboard (k = N for even L) reaches them."""
    L, B = 16, 256
    lo, hi = [0, 200, 240, 250], [210, 245, 252, 256]
    r = O.REWL(0, L, 4, 0.75, 3, 1e-3, 0.8, seed=8, interval=100, prep_budget=2, lo_hi=(lo, hi))
    assert r.init() == 0
    st = r.state()
    for g in range(12):
        w = g // 3
        E = O.energy(0, L, st["spins"][g])
        assert st["k"][g] == (E + 2 * L * L) // 4 and lo[w] <= st["k"][g] <= hi[w]
    assert st["prep_restarts"][9:].sum() > 0  # the top window needed the restart


def test_ising_8x8_config1_shape():
    ex = _exact(0, 8)
    fin = np.isfinite(ex)
    r = O.REWL(0, 8, 4, 0.75, 1, 1e-6, 0.8, seed=0x5EED201400000000 + 1000, interval=10_000)
    assert r.init() == 0
    r.run(10 ** 6)
    out, joins = r.stitch(0)
    st = r.state()
    assert np.all(st["finished"] == 1)
    err = np.abs(out[fin] - ex[fin]).max()
    assert err < 0.5  # one walker per window: WL error saturates at O(0.1)
    acc = st["swap_acc"][:3] / st["swap_att"][:3]
    assert np.all((acc > 0.2) & (acc < 0.9))
    assert all(r.lo[w + 1] <= joins[w] <= r.hi[w] for w in range(3))


def test_detailed_balance_of_moves_and_exchanges():
    """Windows with fixed, window-specific ln g: stationary histograms follow exp(-tilt).

    With ln g_w(k) = ln g(k) + t_w k and ln f ~ 0, the WL move rule samples bin k of window
    w with weight g(k) / g_w(k) = exp(-t_w k).  An exchange rule that breaks detailed
    balance (wrong sign, missing term, swapped operand) distorts these histograms.
    """
    L, h, m = 4, 2, 2
    ex = np.array(X.exact_lng(0, L))
    fin = np.isfinite(ex)
    tilt = [0.15, -0.2]
    # flatness 2.0 is never reached, so ln g stays put (ln f = 1e-13 is negligible)
    r2 = O.REWL(0, L, h, 0.75, m, 1e-14, 2.0, seed=77, interval=3, lnf_init=1e-13)
    lo, hi, W = r2.lo, r2.hi, r2.W
    lng = np.zeros((h * m, W))
    for g in range(h * m):
        w = g // m
        ks = np.arange(lo[w], hi[w] + 1)
        lng[g, : len(ks)] = np.where(fin[ks], ex[np.where(fin[ks], ks, 0)], 0.0) + tilt[w] * ks
    assert r2.init() == 0
    r2.put(lng=lng)
    r2.run(120_000)
    st = r2.state()
    assert np.all(st["swap_acc"][:1] > 1000)
    for w in range(h):
        ks = np.arange(lo[w], hi[w] + 1)
        Hs = st["H"][w * m:(w + 1) * m, : len(ks)].sum(axis=0).astype(float)
        valid = fin[ks]
        p = np.exp(-tilt[w] * ks) * valid
        p /= p.sum()
        n = Hs.sum()
        chi2 = (((Hs - n * p) ** 2) / np.where(valid, n * p, 1.0))[valid].sum()
        dof = valid.sum() - 1
        # visits are correlated (moves change k by at most 2); allow a wide but finite band
        assert chi2 / dof < 40, (w, chi2, dof)
        # the mean bin must match exp(-tilt) weighting closely
        kbar = (Hs * ks).sum() / n
        kexp = (p * ks).sum()
        assert abs(kbar - kexp) < 0.05 * (hi[w] - lo[w]), (w, kbar, kexp)


def test_stitch_reproduces_exact_windows():
    ex = np.array(X.exact_lng(0, 8))
    fin = np.isfinite(ex)
    B, h = 64, 4
    lo, hi = O.windows(B, h, 0.75)
    W = int((hi - lo).max() + 1)
    lngw = np.zeros((h, W))
    valid = np.zeros((h, W), np.uint8)
    rng = np.random.default_rng(3)
    for w in range(h):
        ks = np.arange(lo[w], hi[w] + 1)
        off = rng.normal(0, 50)
        lngw[w, : len(ks)] = np.where(fin[ks], ex[np.where(fin[ks], ks, 0)], 0) + off
        valid[w, : len(ks)] = fin[ks]
    out, joins = O.stitch(0, 8, lo, hi, lngw, valid, norm=0)
    want = X.normalise_lng(ex, 64 * math.log(2))
    assert np.array_equal(np.isfinite(out), fin)
    assert np.abs(out[fin] - want[fin]).max() < 1e-11
    out1, _ = O.stitch(0, 8, lo, hi, lngw, valid, norm=1)
    assert out1[0] == pytest.approx(math.log(2), abs=1e-12)
    assert np.abs((out1 - out1[0])[fin] - (ex - ex[0])[fin]).max() < 1e-11


def test_stitch_picks_bin_where_derivatives_agree():
    # window 1 = window 0 + c (k - k0)^2: the 5-point stencil is exact on quadratics,
    # so |beta_0 - beta_1| = 2c|k - k0|/dE vanishes exactly at k0
    B, h = 64, 2
    lo, hi = O.windows(B, h, 0.75)
    W = int((hi - lo).max() + 1)
    base = np.sin(np.arange(B + 1) * 0.1) * 20 + np.arange(B + 1) * 0.3
    lngw = np.zeros((h, W))
    valid = np.zeros((h, W), np.uint8)
    k0 = 30
    for w in range(h):
        ks = np.arange(lo[w], hi[w] + 1)
        lngw[w, : len(ks)] = base[ks] + (0.01 * (ks - k0) ** 2 if w == 1 else 0)
        valid[w, : len(ks)] = 1
    out, joins = O.stitch(0, 8, lo, hi, lngw, valid, norm=1)
    assert list(joins) == [k0]


def _frag_setup(m=6, L=6, h=3):
    """Exact 6x6 ln g cut into windows, one fragment row per walker."""
    ex = _exact(0, L)
    B = L * L
    lo, hi = O.windows(B, h, 0.75)
    W = int((hi - lo).max()) + 1
    base = np.zeros((h * m, W))
    mask = np.zeros((h, W), np.uint8)
    for w in range(h):
        nb = hi[w] - lo[w] + 1
        seg = ex[lo[w]: hi[w] + 1]
        mask[w, :nb] = np.isfinite(seg)
        for i in range(m):
            base[w * m + i, :nb] = np.where(np.isfinite(seg), seg, 0.0)
    return ex, lo, hi, W, base, mask


def test_jackknife_invariants():
    """Identical fragments: zero error.  A constant offset per walker (a relative density of
    states carries no absolute level): zero error.  Small perturbations: error linear in
    their size."""
    m = 6
    ex, lo, hi, W, base, mask = _frag_setup(m)
    fin = np.isfinite(ex)
    assert np.nanmax(np.abs(O.jackknife(0, 6, lo, hi, base, mask, m))) < 1e-12
    rng = np.random.default_rng(1)
    off = base + rng.normal(0, 3, (base.shape[0], 1))
    assert np.nanmax(np.abs(O.jackknife(0, 6, lo, hi, off, mask, m))) < 1e-10
    z = rng.normal(0, 1, base.shape)
    e1 = O.jackknife(0, 6, lo, hi, base + 1e-6 * z, mask, m)
    e2 = O.jackknife(0, 6, lo, hi, base + 2e-6 * z, mask, m)
    assert np.all(e1[fin] > 0)
    np.testing.assert_allclose(e2[fin], 2 * e1[fin], rtol=1e-4)


def test_jackknife_of_a_linear_statistic_is_the_standard_error():
    """One window (nothing to join); only a bin of negligible weight varies between walkers,
    so the joined ln g there is the plain walker mean, and the jackknife error must be the
    textbook standard error of a mean, s / sqrt(m)."""
    m, L = 8, 6
    ex = _exact(0, L)
    B = L * L
    lo, hi = np.array([0]), np.array([B])
    frag = np.tile(np.where(np.isfinite(ex), ex, 0.0), (m, 1))
    mask = np.isfinite(ex).astype(np.uint8)[None, :]
    b = 0  # the ground state: g = 2 out of 2^36
    d = np.random.default_rng(4).normal(0, 1e-3, m)
    frag[:, b] += d
    err = O.jackknife(0, L, lo, hi, frag, mask, m)
    assert err[b] == pytest.approx(np.std(d, ddof=1) / np.sqrt(m), rel=1e-6)
