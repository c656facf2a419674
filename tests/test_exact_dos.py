"""The exact densities of states pinned to each other and to closed-form facts."""
import math
import os

import numpy as np
import pytest

from oracle import exact_dos as X


def _read(golden_dir, name):
    ks, vs = [], []
    with open(os.path.join(golden_dir, name)) as f:
        for line in f:
            if line.startswith("#"):
                continue
            a, b = line.split()
            ks.append(int(a))
            vs.append(b)
    return ks, vs


def test_three_routes_agree_4x4():
    bf = X.brute_force_ising(4)
    assert bf == X.transfer_matrix_ising(4) == X.kaufman_ising(4)
    assert sum(bf) == 2 ** 16


def test_transfer_matrix_equals_kaufman_6x6():
    assert X.transfer_matrix_ising(6) == X.kaufman_ising(6)


@pytest.mark.parametrize("L", [4, 6, 8, 10, 12, 16])
def test_ising_invariants(L):
    N = L * L
    g = X.kaufman_ising(L)
    assert len(g) == N + 1 and sum(g) == 2 ** N
    assert g[0] == 2 and g[1] == 0  # ground states; one broken bond pair impossible
    assert g[2] == 2 * N  # one flipped spin: 4 broken bonds
    assert g[3] == 4 * N  # two adjacent flipped spins: 6 broken bonds
    if L >= 6:
        assert g[4] == N * (N + 9)
    assert g == g[::-1]  # E <-> -E for even L (sublattice flip)
    assert g[-2] == 0 and g[-1] == 2


def test_golden_L8_counts(golden_dir):
    ks, vs = _read(golden_dir, "ising_L8_counts.txt")
    assert [int(v) for v in vs] == X.kaufman_ising(8)


@pytest.mark.parametrize("L", [16, 32])
def test_golden_lng_files_match_closed_form(golden_dir, L):
    ks, vs = _read(golden_dir, f"ising_L{L}_lng.txt")
    got = np.array([float(v) for v in vs])
    want = X.ln_of_counts(X.kaufman_ising(L))
    assert np.array_equal(np.isfinite(got), np.isfinite(want))
    fin = np.isfinite(want)
    assert np.max(np.abs(got[fin] - want[fin])) < 1e-12


def test_golden_L64_invariants(golden_dir):
    ks, vs = _read(golden_dir, "ising_L64_lng.txt")
    N = 64 * 64
    lng = np.array([float(v) for v in vs])
    assert len(lng) == N + 1
    assert lng[0] == pytest.approx(math.log(2), abs=1e-15)
    assert lng[1] == -np.inf and lng[N - 1] == -np.inf
    assert lng[2] == pytest.approx(math.log(2 * N), abs=1e-13)
    assert lng[3] == pytest.approx(math.log(4 * N), abs=1e-13)
    assert lng[4] == pytest.approx(math.log(N * (N + 9)), abs=1e-13)
    fin = np.isfinite(lng)
    assert np.allclose(lng[fin], lng[::-1][fin], rtol=0, atol=1e-9)
    mx = lng[fin].max()
    assert mx + math.log(np.exp(lng[fin] - mx).sum()) == pytest.approx(N * math.log(2), rel=1e-13)


def test_potts_q3_3x3():
    g = X.brute_force_potts(3, 3)
    N, q = 9, 3
    assert sum(g) == q ** N
    assert g[0] == q
    assert g[1] == g[2] == g[3] == 0
    assert g[4] == N * q * (q - 1)  # one site changed: 4 broken bonds


def test_potts_q2_is_ising():
    gp = X.brute_force_potts(4, 2)
    gi = X.brute_force_ising(4)
    assert gp[0::2] == gi and not any(gp[1::2])
