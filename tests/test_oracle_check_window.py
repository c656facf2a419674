"""Pins of the oracle's flatness test and window advance (Sec. 2), on hand-built windows.

Sec. 2: a walker's histogram is "flat" when its smallest entry reaches a fixed fraction (0.8)
of its mean; when all m walkers of a window are flat, their estimates of ln g are combined and
handed back to every walker, H is reset and ln f is halved (f -> sqrt f).  Readings:
  * flat  <=>  min H * count >= flatness * sum H over the bins any walker of the window has
    visited so far (cumulative over iterations); the flag latches until the window advances;
  * the combination is the ln-domain mean over walkers 0..m-1, summed in that order;
  * a window runs while ln f >= ln f_final; the 1/t variant sets ln f = visited bins / moves.
Each case is built so that a plausible slip (">" for ">=", walker 0's ln g instead of the mean,
a log-mean-exp, another summation order, a mask limited to this iteration, a flag that does not
latch, a missing H reset) changes the outcome.  Expected values are worked out by hand.
"""
import numpy as np
import pytest

import oracle as O

# Ising 4x4, one window over all 17 bins, three walkers
M = 3


def make(lnf_init=1.0, lnf_final=1e-8, schedule=0, flatness=0.8):
    o = O.REWL(0, 4, 1, 0.75, M, lnf_final, flatness, seed=1, interval=100, lnf_init=lnf_init,
               schedule=schedule)
    assert (o.h, o.m, o.W) == (1, M, 17)
    return o


def plant(o, H_rows, lng_rows=None, step=1000, **win):
    H = np.zeros((M, o.W), np.uint32)
    for i, row in enumerate(H_rows):
        H[i, : len(row)] = row
    lng = np.zeros((M, o.W), np.float64)
    if lng_rows is not None:
        for i, row in enumerate(lng_rows):
            lng[i, : len(row)] = row
    o.put(lng=lng, H=H, step=np.full(M, step, np.uint64))
    if win:
        o.put_window(**win)
    return H, lng


FLAT = [4, 5, 5, 5, 6]      # min*count = 20 = 0.8 * 25: flat exactly at the threshold
UNFLAT = [4, 5, 5, 5, 7]    # one count more: 20 < 0.8 * 26


def test_flag_exactly_at_threshold_and_one_count_below():
    o = make()
    H, lng = plant(o, [FLAT, UNFLAT, FLAT])
    o.check(0)
    s = o.state()
    assert s["flat"].tolist() == [1, 0, 1]
    # no advance while a walker is not flat
    assert s["lnf"][0] == 1.0 and s["iter"][0] == 0
    assert np.array_equal(s["H"], H) and np.array_equal(s["lng"], lng)
    # the valid mask is the union of the visited bins
    assert s["mask"][0].tolist() == [1] * 5 + [0] * 12


def test_bin_visited_by_another_walker_counts():
    o = make()
    other = FLAT + [1]          # walker 1 visited bin 5, walker 0 never did: min H = 0 there
    plant(o, [FLAT, other, other])
    o.check(0)
    s = o.state()
    assert s["flat"].tolist() == [0, 0, 0]
    assert s["mask"][0, :6].tolist() == [1] * 6


def test_mask_is_cumulative_over_iterations():
    o = make()
    mask = np.zeros((1, o.W), np.uint8)
    mask[0, 9] = 1              # visited in an earlier iteration, not in this one
    plant(o, [FLAT, FLAT, FLAT], mask=mask)
    o.check(0)
    s = o.state()
    assert s["flat"].tolist() == [0, 0, 0] and s["iter"][0] == 0
    assert s["mask"][0].tolist() == [1] * 5 + [0] * 4 + [1] + [0] * 7


def test_flag_latches_until_the_window_advances():
    o = make()
    # walker 0 was found flat at an earlier check; its histogram has since become uneven
    plant(o, [[0, 9, 9, 9, 9], FLAT, FLAT], flat=np.array([1, 0, 0], np.uint8))
    o.check(0)
    s = o.state()
    assert s["iter"][0] == 1, "a latched flag must count towards the advance"
    assert s["flat"].tolist() == [0, 0, 0]


def test_advance_is_the_ln_domain_mean_in_walker_order():
    o = make()
    lng_rows = [[0.1, 1.0, -3.0, 7.5, 100.0],
                [0.2, 2.0, -3.0, 7.5, 100.0],
                [0.3, 4.0, -3.0, 7.5, 100.0]]
    plant(o, [FLAT, FLAT, FLAT], lng_rows, round=41)
    o.check(0)
    s = o.state()
    # bin 0: ((0.1 + 0.2) + 0.3) / 3 in float64 = 0x1.999999999999bp-3; the reverse order would
    # give 0.19999999999999998
    assert s["lng"][:, 0].tolist() == [float.fromhex("0x1.999999999999bp-3")] * M
    # bin 1: 7/3 (log-mean-exp of e, e^2, e^4 would be 3.0712..., walker 0 alone 1.0)
    assert s["lng"][:, 1].tolist() == [2.3333333333333335] * M
    assert s["lng"][:, 2:5].tolist() == [[-3.0, 7.5, 100.0]] * M
    assert not s["H"].any() and s["flat"].tolist() == [0, 0, 0]
    assert s["lnf"][0] == 0.5 and s["iter"][0] == 1 and s["finished"][0] == 0
    assert s["first_iter_round"][0] == 42 and s["mode"][0] == 0
    assert s["mask"][0].tolist() == [1] * 5 + [0] * 12


def test_last_halving_finishes_and_keeps_fragments():
    lnf = 2.0 ** -26             # 1.49e-8 >= 1e-8: still running; half of it is below 1e-8
    o = make(lnf_init=lnf)
    rows = [[1.0, 2.0, 3.0, 4.0, 5.0], [1.5, 2.5, 3.5, 4.5, 5.5], [2.0, 3.0, 4.0, 5.0, 6.0]]
    plant(o, [FLAT, FLAT, FLAT], rows, iter=np.array([26], np.int32))
    o.check(0)
    s = o.state()
    assert s["lnf"][0] == 2.0 ** -27 and s["finished"][0] == 1 and s["iter"][0] == 27
    assert s["frag"][:, :5].tolist() == rows
    assert s["lng"][:, :5].tolist() == [[1.5, 2.5, 3.5, 4.5, 5.5]] * M
    # a finished window is not checked again
    plant(o, [FLAT, FLAT, FLAT], rows)
    o.check(0)
    assert o.state()["H"][:, :5].tolist() == [FLAT] * M


def test_not_finished_at_exactly_lnf_final():
    o = make(lnf_init=2.0 ** -9, lnf_final=2.0 ** -10)
    plant(o, [FLAT, FLAT, FLAT])
    o.check(0)
    s = o.state()
    assert s["lnf"][0] == 2.0 ** -10 and s["finished"][0] == 0


@pytest.mark.parametrize("step,switch", [(5000, True), (20000, False)])
def test_one_over_t_switch(step, switch):
    # after the halving ln f = 2^-11 = 4.88e-4; 1/t = visited bins / moves = 5 / step
    o = make(lnf_init=2.0 ** -10, schedule=1)
    plant(o, [FLAT, FLAT, FLAT], step=step)
    o.check(0)
    s = o.state()
    if switch:
        assert s["mode"][0] == 1 and s["lnf"][0] == 0.001
    else:
        assert s["mode"][0] == 0 and s["lnf"][0] == 2.0 ** -11


def test_one_over_t_mode_averages_without_flatness():
    o = make(lnf_init=0.001, schedule=1)
    rows = [[0.0, 1.0, 0.0, 0.0, 0.0], [0.0, 2.0, 0.0, 0.0, 0.0], [0.0, 3.0, 0.0, 0.0, 0.0]]
    plant(o, [UNFLAT, [0, 9, 9, 9, 9], UNFLAT], rows, step=10000,
          mode=np.array([1], np.uint8), iter=np.array([12], np.int32))
    o.check(0)
    s = o.state()
    assert s["lnf"][0] == 0.0005 and s["iter"][0] == 13 and s["mode"][0] == 1
    assert s["lng"][:, 1].tolist() == [2.0] * M and not s["H"].any()
