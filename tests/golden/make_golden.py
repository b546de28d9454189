"""Writes the stored exact values under tests/golden/.  Calls only oracle/.

Usage: python tests/golden/make_golden.py
"""
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402


def main():
    L, N = 8, 64
    om = oracle.tm_ising(L)
    with open(os.path.join(HERE, "ising_L8_omega.txt"), "w") as f:
        f.write("# Exact density of states Omega(E) of the 8x8 periodic Ising model (J = 1),\n")
        f.write("# H = -J sum_<ij> s_i s_j (Ising paragraph of the paper); this is the table Beale\n")
        f.write("# (PRL 76, 78 (1996)) published, recomputed here by the oracle's transfer matrix,\n")
        f.write("# which tests/test_oracle_exact.py pins to Kaufman's closed form.\n")
        f.write("# columns: E  Omega(E)\n")
        for j, o in enumerate(om):
            f.write("%d %d\n" % (4 * j - 2 * N, o))


if __name__ == "__main__":
    main()
