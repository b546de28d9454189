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

    # 4 x 4 q = 8 Potts (the benchmark's q; the proposal draws from q - 1 = 7 colours)
    L, q, N = 4, 8, 16
    om = oracle.tm_potts(L, q)
    with open(os.path.join(HERE, "potts_q8_L4_omega.txt"), "w") as f:
        f.write("# Exact density of states Omega(E) of the 4x4 periodic q = 8 Potts model (J = 1),\n")
        f.write("# H = -J sum_<ij> delta(s_i, s_j) (Potts paragraph of the paper), by the oracle's transfer\n")
        f.write("# matrix, which tests/test_oracle_exact.py pins to brute force (q = 3) and to counting.\n")
        f.write("# columns: E  Omega(E)\n")
        for j, o in enumerate(om):
            f.write("%d %d\n" % (j - 2 * N, o))

    # 16 x 16 and 32 x 32: thermodynamics from Kaufman's closed form (oracle/exact.py), the derivatives of ln Z
    # by central differences at 60 digits (step 1e-12 / 1e-10, truncation ~1e-20):
    # <E> = -d lnZ / d beta, C = beta^2 d^2 lnZ / d beta^2.
    import mpmath

    from oracle import exact

    for L in (16, 32):
        _kaufman_table(L, mpmath, exact)


def _kaufman_table(L, mpmath, exact):
    N = L * L
    with mpmath.workdps(60):
        with open(os.path.join(HERE, "ising_L%d_kaufman.txt" % L), "w") as f:
            f.write("# Exact thermodynamics of the %dx%d periodic Ising model (J = 1), from Kaufman's\n" % (L, L))
            f.write("# closed form of Z (Phys. Rev. 76, 1232 (1949)) as evaluated by oracle/exact.py;\n")
            f.write("# <E> = -d lnZ/d beta and C = beta^2 d^2 lnZ/d beta^2 by central differences at 60 digits.\n")
            f.write("# columns: beta  lnZ  <E>/N  C/N\n")
            for beta in ("0.2", "0.3", "0.4", "0.4406867935097715", "0.5", "0.6"):
                b = mpmath.mpf(beta)
                lz = lambda t: exact.kaufman_lnZ(L, L, t)  # noqa: E731
                lnZ = lz(b)
                h1, h2 = mpmath.mpf("1e-12"), mpmath.mpf("1e-10")
                d1 = (lz(b + h1) - lz(b - h1)) / (2 * h1)
                d2 = (lz(b + h2) - 2 * lnZ + lz(b - h2)) / (h2 * h2)
                f.write("%s %s %s %s\n" % (beta, mpmath.nstr(lnZ, 20), mpmath.nstr(-d1 / N, 20),
                                            mpmath.nstr(b * b * d2 / N, 20)))


if __name__ == "__main__":
    main()
