"""Writes the exact density-of-states fixtures in this folder.

Every value comes from ``oracle.exact_dos`` (enumeration, transfer matrix,
Kaufman/Beale).  Run from the repository root:  python tests/golden/make_golden.py
"""
import math
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import exact_dos as X  # noqa: E402


def write_counts(name, counts, header):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {header}\n# k g_k (exact integer)\n")
        for k, v in enumerate(counts):
            f.write(f"{k} {v}\n")


def write_lng(name, lng, header):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {header}\n# k ln g_k (-inf where g_k = 0)\n")
        for k, v in enumerate(lng):
            f.write(f"{k} {float(v)!r}\n")


def write_em(name, g, header):
    with open(os.path.join(HERE, name), "w") as f:
        f.write(f"# {header}\n# k j g(k, j) (exact integer; k = E/4 + N/2, j = (M + N)/2; "
                f"zero entries omitted)\n")
        for k in range(g.shape[0]):
            for j in range(g.shape[1]):
                if g[k, j]:
                    f.write(f"{k} {j} {int(g[k, j])}\n")


def main():
    bf4 = X.brute_force_ising(4)
    assert bf4 == X.kaufman_ising(4) == X.transfer_matrix_ising(4)
    write_counts("ising_L4_counts.txt", bf4,
                 "2D Ising 4x4 periodic, enumeration of 2^16 states (= Kaufman = transfer matrix)")
    tm8 = X.transfer_matrix_ising(8)
    ka8 = X.kaufman_ising(8)
    assert tm8 == ka8 and sum(ka8) == 2 ** 64
    write_counts("ising_L8_counts.txt", ka8,
                 "2D Ising 8x8 periodic, Kaufman/Beale closed form, equal to the transfer matrix")
    p3 = X.brute_force_potts(3, 3)
    assert sum(p3) == 3 ** 9
    write_counts("potts_q3_L3_counts.txt", p3, "2D q=3 Potts 3x3 periodic, enumeration of 3^9 states")
    em4 = X.brute_force_ising_em(4)
    assert (em4 == X.transfer_matrix_ising_em(4)).all()
    em6 = X.transfer_matrix_ising_em(6)
    assert [int(v) for v in em6.sum(axis=1)] == X.transfer_matrix_ising(6)
    assert (em6 == em6[:, ::-1]).all()
    write_em("ising_L6_em_counts.txt", em6,
             "2D Ising 6x6 periodic, joint g(E, M) by the (E, M) transfer matrix; sums over M "
             "equal the 1D transfer matrix, symmetric under M -> -M")
    for L in (16, 32, 64):
        g = X.kaufman_ising(L)
        assert sum(g) == 2 ** (L * L)
        write_lng(f"ising_L{L}_lng.txt", X.ln_of_counts(g),
                  f"2D Ising {L}x{L} periodic, Kaufman/Beale closed form, sum g = 2^{L * L} checked")


if __name__ == "__main__":
    main()
