"""Pins of the CPU oracle's building blocks against facts that do not come from it.

Every check here would fail on a plausible slip in the oracle (a dropped term, a
wrong sign, index or operand order), and none retypes the oracle's own formula.
"""
import math

import numpy as np
import pytest

import oracle as O
from oracle import exact_dos as X
from tests import inputs as I


# ---------------------------------------------------------------- Philox4x32-10
# Known-answer vectors published with the Random123 library of Salmon, Moraes,
# Dror and Shaw (SC'11, "Parallel random numbers: as easy as 1, 2, 3"),
# philox4x32 with 10 rounds.
KAT = [
    ((0, 0, 0, 0), (0, 0), (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)),
    ((0xFFFFFFFF,) * 4, (0xFFFFFFFF,) * 2, (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)),
    ((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0),
     (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)),
]


@pytest.mark.parametrize("ctr,key,expect", KAT)
def test_philox_known_answers(ctr, key, expect):
    assert tuple(int(v) for v in O.philox(ctr, key)) == expect


def test_philox_words_look_uniform():
    # 4 * 20000 words: mean of top byte and bit balance within 5 sigma
    words = np.concatenate([O.philox((i, 7, 3, 0), (11, 13)) for i in range(20000)])
    bits = ((words[:, None] >> np.arange(32, dtype=np.uint32)) & 1).mean(axis=0)
    assert np.all(np.abs(bits - 0.5) < 5 * 0.5 / math.sqrt(len(words)))


# ---------------------------------------------------------------- ln u
def test_lnu_matches_libm_within_4_ulp():
    rng = np.random.default_rng(5)
    ws = np.concatenate([rng.integers(0, 2 ** 32, 50000), np.arange(0, 64),
                         2 ** 32 - 1 - np.arange(0, 64), 2 ** np.arange(0, 32)])
    for w in ws:
        exact = math.log((int(w) + 0.5) / 2 ** 32)
        got = O.lnu(int(w))
        assert abs(got - exact) <= 4 * math.ulp(exact), (w, got, exact)
        assert got < 0.0


def test_lnu_endpoints_and_monotone():
    assert O.lnu(0) == pytest.approx(-33 * math.log(2), abs=1e-14)
    assert O.lnu(2 ** 31) == pytest.approx(math.log(0.5 + 2 ** -33), abs=1e-15)
    assert -1.2e-10 < O.lnu(2 ** 32 - 1) < 0.0
    rng = np.random.default_rng(9)
    ws = np.sort(rng.integers(0, 2 ** 32, 20000))
    vals = np.array([O.lnu(int(w)) for w in ws])
    assert np.all(np.diff(vals) >= 0.0)


# ---------------------------------------------------------------- windows (Fig. 1a)
def test_windows_config1_by_hand():
    # B = 64 bins, h = 4, o = 3/4: W = 4B/(h+3) = 36.57, step s = B/(h+3) = 9.14
    # lo = round(k s) = 0, 9, 18, 27; hi = round(k s + W) = 37, 46, 55, 64
    lo, hi = O.windows(64, 4, 0.75)
    assert list(lo) == [0, 9, 18, 27] and list(hi) == [37, 46, 55, 64]


@pytest.mark.parametrize("B,h,o", [(4096, 32, 0.75), (3200, 64, 0.75), (12800, 64, 0.75),
                                   (256, 8, 0.75), (1000, 7, 0.5), (64, 1, 0.75), (500, 5, 0.6)])
def test_windows_cover_and_overlap(B, h, o):
    lo, hi = O.windows(B, h, o)
    assert lo[0] == 0 and hi[-1] == B
    W = B / (1 + (h - 1) * (1 - o))
    for k in range(h):
        assert abs(lo[k] - k * (1 - o) * W) <= 0.5 + 1e-9
        if k < h - 1:
            assert abs(hi[k] - (k * (1 - o) * W + W)) <= 0.5 + 1e-9
            ov = hi[k] - lo[k + 1]
            assert abs(ov - o * W) <= 1.0 + 1e-9  # overlap fraction o of a window
    # every bin lies in at least one window
    cov = np.zeros(B + 1, bool)
    for a, b in zip(lo, hi):
        cov[a:b + 1] = True
    assert cov.all()


def test_windows_reject_no_overlap():
    with pytest.raises(ValueError):
        O.windows(10, 20, 0.75)


# ---------------------------------------------------------------- energies
@pytest.mark.parametrize("L", [3, 4, 5, 8])
def test_energy_extremes(L):
    N = L * L
    assert O.energy(0, L, np.ones(N, np.int8)) == -2 * N
    assert O.energy(3, L, np.zeros(N, np.int8)) == -2 * N
    s = np.ones(N, np.int8)
    s[L + 1] = -1
    assert O.energy(0, L, s) == -2 * N + 8  # one flipped spin breaks 4 bonds, 2 each
    p = np.zeros(N, np.int8)
    p[L + 1] = 2
    assert O.energy(3, L, p) == -2 * N + 4
    if L % 2 == 0:
        cb = np.array([1 if (x + y) % 2 == 0 else -1 for y in range(L) for x in range(L)], np.int8)
        assert O.energy(0, L, cb) == 2 * N
    # Potts with all neighbours different: colour (x + 2y) mod 5 for L multiple of 5
    if L % 5 == 0:
        c = np.array([(x + 2 * y) % 5 for y in range(L) for x in range(L)], np.int8)
        assert O.energy(5, L, c) == 0


def test_energy_histogram_equals_exact_counts_4x4():
    # route every 4x4 configuration through the oracle's energy; compare with the
    # Kaufman closed form
    N = 16
    counts = np.zeros(N + 1, np.int64)
    idx = np.arange(1 << N)
    spins = ((idx[:, None] >> np.arange(N)) & 1).astype(np.int8) * 2 - 1
    for s in spins:
        E = O.energy(0, 4, s)
        counts[(E + 2 * N) // 4] += 1
    assert list(counts) == X.kaufman_ising(4)


# ---------------------------------------------------------------- one WL move (Sec. 2)
def _move_case(model, L, n, seed, lnf=0.25, frozen=False, scale=3.0):
    rng = np.random.default_rng(seed)
    N = L * L
    q = 2 if model == 0 else model
    B = O.num_bins(model, L)
    spins = I.random_lattices(rng, model, L, n)
    k = np.array([(O.energy(model, L, s) + 2 * N) // (4 if model == 0 else 1) for s in spins],
                 np.int32)
    # windows around the current bin, sometimes tight so that proposals fall outside
    lo = np.maximum(0, k - rng.integers(0, 6, n)).astype(np.int32)
    hi = np.minimum(B, k + rng.integers(0, 6, n)).astype(np.int32)
    W = 16
    lng = I.random_lng(rng, n, W, scale=scale)
    H = I.random_H(rng, n, W)
    words = I.random_words(rng, n)
    res = O.replay_batch(model, q, L, spins, k, lo, hi, lng, H, np.full(n, lnf),
                         np.full(n, frozen, np.uint8), words)
    return dict(spins=spins, k=k, lo=lo, hi=hi, lng=lng, H=H, words=words, q=q, N=N), res


@pytest.mark.parametrize("model,L", [(0, 4), (0, 7), (0, 8), (3, 5), (10, 6), (2, 4)])
def test_move_energy_bookkeeping(model, L):
    inp, res = _move_case(model, L, 400, seed=L * 31 + model)
    N, q = inp["N"], inp["q"]
    for i in range(400):
        s0, s1 = inp["spins"][i], res["spins"][i]
        changed = np.flatnonzero(s0 != s1)
        E1 = O.energy(model, L, s1)
        kb = (E1 + 2 * N) // (4 if model == 0 else 1)
        assert res["k"][i] == kb  # the tracked bin is the bin of the new configuration
        site = (int(inp["words"][i, 0]) * N) >> 32
        if res["acc"][i]:
            assert list(changed) == [site]
            if model != 0:
                r = (int(inp["words"][i, 1]) * (q - 1)) >> 32
                assert s1[site] == (s0[site] + 1 + r) % q and s1[site] != s0[site]
            # dk reported is the energy change of the flip (in bins)
            assert res["dk"][i] == kb - inp["k"][i]
        else:
            assert len(changed) == 0 and res["k"][i] == inp["k"][i]


@pytest.mark.parametrize("model,L", [(0, 8), (10, 6)])
def test_move_acceptance_rule(model, L):
    # min[1, g(E_old)/g(E_new)] with ln u computed by libm, not the oracle's log
    inp, res = _move_case(model, L, 3000, seed=77 + model, scale=0.7)
    for i in range(3000):
        k0, dk = int(inp["k"][i]), int(res["dk"][i])
        lo, hi = int(inp["lo"][i]), int(inp["hi"][i])
        kp = k0 + dk
        if not (lo <= kp <= hi):
            assert res["acc"][i] == 0  # outside the window: rejected
            continue
        d = inp["lng"][i, k0 - lo] - inp["lng"][i, kp - lo]
        lnu = math.log((int(inp["words"][i, 2]) + 0.5) / 2 ** 32)
        if abs(lnu - d) < 1e-12:
            continue
        assert res["acc"][i] == int(lnu < d), (i, d, lnu)


def test_move_updates_lng_and_H_at_new_bin():
    inp, res = _move_case(0, 8, 500, seed=3, lnf=0.125)
    for i in range(500):
        lo = int(inp["lo"][i])
        b = int(res["k"][i]) - lo
        d_lng = res["lng"][i] - inp["lng"][i]
        d_H = res["H"][i].astype(np.int64) - inp["H"][i]
        assert d_H[b] == 1 and d_H.sum() == 1
        assert res["lng"][i, b] == inp["lng"][i, b] + 0.125
        assert np.count_nonzero(d_lng) == 1


def test_move_frozen_window_keeps_lng_and_H():
    inp, res = _move_case(0, 8, 300, seed=4, frozen=True)
    assert np.array_equal(res["lng"], inp["lng"]) and np.array_equal(res["H"], inp["H"])
    assert res["acc"].sum() > 0


def test_potts_proposal_uniform_over_other_states():
    q, L, n = 10, 4, 20000
    rng = np.random.default_rng(12)
    spins = np.zeros((n, L * L), np.int8)  # all state 0
    k = np.zeros(n, np.int32)
    words = I.random_words(rng, n)
    words[:, 2] = 0  # ln u minimal: accept whenever inside the window
    res = O.replay_batch(q, q, L, spins, k, np.zeros(n, np.int32), np.full(n, 32, np.int32),
                         np.zeros((n, 33)), np.zeros((n, 33), np.uint32), np.full(n, 0.1),
                         np.zeros(n, np.uint8), words)
    assert res["acc"].all()
    new = res["spins"].max(axis=1)
    counts = np.bincount(new, minlength=q)
    assert counts[0] == 0
    exp = n / (q - 1)
    chi2 = ((counts[1:] - exp) ** 2 / exp).sum()
    assert chi2 < 30  # 8 dof


def test_site_choice_uniform():
    L, n = 5, 25000
    rng = np.random.default_rng(2)
    spins = np.ones((n, L * L), np.int8)
    words = I.random_words(rng, n)
    words[:, 2] = 0
    res = O.replay_batch(0, 2, L, spins, np.zeros(n, np.int32), np.zeros(n, np.int32),
                         np.full(n, 25, np.int32), np.zeros((n, 26)),
                         np.zeros((n, 26), np.uint32), np.full(n, 0.1), np.zeros(n, np.uint8),
                         words)
    sites = np.argmin(res["spins"], axis=1)
    counts = np.bincount(sites, minlength=L * L)
    exp = n / (L * L)
    assert ((counts - exp) ** 2 / exp).sum() < 60  # 24 dof
