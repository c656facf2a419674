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
    for L in (16, 32, 64):
        g = X.kaufman_ising(L)
        assert sum(g) == 2 ** (L * L)
        write_lng(f"ising_L{L}_lng.txt", X.ln_of_counts(g),
                  f"2D Ising {L}x{L} periodic, Kaufman/Beale closed form, sum g = 2^{L * L} checked")


if __name__ == "__main__":
    main()
