"""Pins of the oracle's replica exchange (Sec. 2, Eq. 1) on hand-built two-window states.

Eq. (1): a configuration X of walker i (window w) and Y of walker j (window w+1) swap with
probability min(1, g_i(E_X) g_j(E_Y) / (g_i(E_Y) g_j(E_X))), impossible when an energy lies
outside the other window.  In logs: ln P = (ln g_i(X) - ln g_i(Y)) + (ln g_j(Y) - ln g_j(X)),
accepted iff ln P >= 0 or ln u < ln P.  The ln g rows are chosen so that a swapped sign, a
swapped index or a missing term flips the outcome; u is drawn by Philox (pinned by its
published vectors) with the exchange's counter, and its log taken with libm, far from ln P.
"""
import math

import numpy as np
import pytest

import oracle as O

SEED = 0x1234567890ABCDEF


def _two_windows():
    o = O.REWL(0, 4, 2, 0.75, 1, 1e-6, 0.8, seed=SEED, interval=10)
    assert (o.lo.tolist(), o.hi.tolist()) == ([0, 3], [13, 16])  # overlap 3..13
    return o


def _plant(o, kx, ky, gi, gj):
    """Walker 0 of window 0 holds X (bin kx), walker 0 of window 1 holds Y (bin ky); ln g of
    walker i / j given as {bin: value}; lattices are markers (+1s / -1s)."""
    spins = np.stack([np.ones(16, np.int8), -np.ones(16, np.int8)])
    lng = np.zeros((2, o.W))
    for b, v in gi.items():
        lng[0, b - o.lo[0]] = v
    for b, v in gj.items():
        lng[1, b - o.lo[1]] = v
    o.put(spins=spins, k=np.array([kx, ky], np.int32), lng=lng)


def _lnu(rd):
    # accept draw of pair index i = 0 with m = 1 walkers: counter (m + i, round, window, tag 3)
    w0 = int(O.philox([1, rd, 0, 3], [SEED & 0xFFFFFFFF, SEED >> 32])[0])
    return math.log((w0 + 0.5) * 2.0 ** -32)


def _swapped(o):
    s = o.state()
    return s["k"].tolist(), bool(s["spins"][0, 0] == -1), int(s["swap_att"][0]), int(s["swap_acc"][0])


def test_positive_lnP_always_swaps():
    # (5 - 0) + (-3 - 0) = +2: accepted whatever u; a sign slip in either bracket gives -2 or -8
    o = _two_windows()
    _plant(o, 5, 9, {5: 5.0, 9: 0.0}, {9: -3.0, 5: 0.0})
    rd = next(r for r in range(200) if _lnu(r) > -1.5)  # a draw that would reject ln P = -2
    o.swap(0, rd)
    assert _swapped(o) == ([9, 5], True, 1, 1)


def test_negative_lnP_follows_the_draw():
    # (5 - 0) + (-7 - 0) = -2: accepted iff ln u < -2
    for want in (True, False):
        rd = next(r for r in range(500) if (_lnu(r) < -2.5) == want and abs(_lnu(r) + 2) > 0.5)
        o = _two_windows()
        _plant(o, 5, 9, {5: 5.0, 9: 0.0}, {9: -7.0, 5: 0.0})
        o.swap(0, rd)
        k, moved, att, acc = _swapped(o)
        assert (k == [9, 5]) == want and moved == want and (att, acc) == (1, int(want))


def test_each_term_matters():
    # ln g_i(Y) alone decides: with it +10 the product is e^-10 (rejected for this draw); a
    # version that dropped or transposed that term would accept
    rd = next(r for r in range(500) if _lnu(r) > -5)
    o = _two_windows()
    _plant(o, 5, 9, {5: 0.0, 9: 10.0}, {9: 0.0, 5: 0.0})
    o.swap(0, rd)
    assert _swapped(o)[0] == [5, 9]
    o = _two_windows()
    _plant(o, 5, 9, {5: 0.0, 9: 0.0}, {9: 0.0, 5: 10.0})  # ln g_j(X) = 10: rejected too
    o.swap(0, rd)
    assert _swapped(o)[0] == [5, 9]
    o = _two_windows()
    _plant(o, 5, 9, {5: 0.0, 9: 0.0}, {9: 10.0, 5: 0.0})  # ln g_j(Y) = 10: accepted
    o.swap(0, rd)
    assert _swapped(o)[0] == [9, 5]


@pytest.mark.parametrize("kx,ky", [(1, 9), (2, 9), (5, 15), (5, 14), (0, 16)])
def test_energy_outside_the_other_window_never_swaps(kx, ky):
    # window 0 = [0, 13], window 1 = [3, 16]: X (in window 0) must also lie in window 1 and
    # Y (in window 1) also in window 0, i.e. both in 3..13
    o = _two_windows()
    gi = {b: 0.0 for b in range(0, 14)}
    gj = {b: 0.0 for b in range(3, 17)}
    gi[kx] = 50.0  # would make ln P huge if the exchange were possible
    _plant(o, kx, ky, gi, gj)
    o.swap(0, 3)
    k, moved, att, acc = _swapped(o)
    assert k == [kx, ky] and not moved and (att, acc) == (1, 0)
