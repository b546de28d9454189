"""Exact reference results used to pin the oracle (test infrastructure only).

* ``kaufman_lnZ``: Kaufman's closed form (Phys. Rev. 76, 1232 (1949)) of the
  partition function of the periodic m x n Ising model, evaluated with mpmath.
  It is independent of every enumeration in ``muca_oracle.c`` and pins the
  exact densities of states (Beale's Omega(E) for L = 8 is recomputed by the
  transfer matrix, never typed in).
* ``lnZ_from_omega``: Z(beta) = sum_E Omega(E) exp(-beta E), the definition
  behind Eq. (1) and (2) of the paper.
* ``fene_dimer_omega``: closed form of the binned density of states of two
  beads joined by one FENE bond (no Lennard-Jones term, since that acts only
  on pairs |i-j| >= 2 in Eq. (7)).
"""
from __future__ import annotations

import mpmath


def kaufman_lnZ(m: int, n: int, beta: float, J: float = 1.0, dps: int = 60):
    """ln Z of the m x n torus (m rows, n columns), H = -J sum s_i s_j, nearest neighbours."""
    with mpmath.workdps(dps):
        K = mpmath.mpf(beta) * J
        c = mpmath.cosh(2 * K) / mpmath.tanh(2 * K)

        def gamma(l):
            if l == 0:
                return 2 * K + mpmath.log(mpmath.tanh(K))
            return mpmath.acosh(c - mpmath.cos(mpmath.pi * l / n))

        z1 = z2 = z3 = z4 = mpmath.mpf(1)
        for r in range(n):
            g_odd, g_even = gamma(2 * r + 1), gamma(2 * r)
            z1 *= 2 * mpmath.cosh(m * g_odd / 2)
            z2 *= 2 * mpmath.sinh(m * g_odd / 2)
            z3 *= 2 * mpmath.cosh(m * g_even / 2)
            z4 *= 2 * mpmath.sinh(m * g_even / 2)
        Z = mpmath.mpf(1) / 2 * (2 * mpmath.sinh(2 * K)) ** (mpmath.mpf(m * n) / 2) * (z1 + z2 + z3 + z4)
        return mpmath.log(Z)


def lnZ_from_omega(omega, energies, beta: float, dps: int = 60):
    """ln sum_E Omega(E) exp(-beta E) in high precision (omega: Python ints)."""
    with mpmath.workdps(dps):
        b = mpmath.mpf(beta)
        Z = mpmath.fsum(mpmath.mpf(int(o)) * mpmath.exp(-b * E) for o, E in zip(omega, energies) if o)
        return mpmath.log(Z)


def fene_dimer_omega(e_edges, K: float, R: float, dps: int = 40):
    """Relative binned density of states of a FENE dimer, V(r) = -(K/2) R^2 ln(1 - (r/R)^2).

    The bond vector is uniform in the ball r < R; r(E) = R sqrt(1 - exp(-2E/(K R^2))), so the
    phase-space volume with V < E is (4 pi / 3) r(E)^3 and a bin [E_a, E_b) holds
    (4 pi / 3)(r(E_b)^3 - r(E_a)^3).  Returns the per-bin volumes.
    """
    with mpmath.workdps(dps):
        KR2 = mpmath.mpf(K) * mpmath.mpf(R) ** 2

        def r_of(E):
            E = mpmath.mpf(E)
            if E <= 0:
                return mpmath.mpf(0)
            return mpmath.mpf(R) * mpmath.sqrt(1 - mpmath.exp(-2 * E / KR2))

        vols = []
        for a, b in zip(e_edges[:-1], e_edges[1:]):
            vols.append(float(4 * mpmath.pi / 3 * (r_of(b) ** 3 - r_of(a) ** 3)))
        return vols


def fene_shifted_dimer_omega(e_edges, K: float, R: float, r0: float, dps: int = 40):
    """Relative binned density of states of a FENE dimer with rest length r0 (the paper's
    Eq. 7 bond), V(r) = -(K/2) R^2 ln(1 - ((r - r0)/R)^2) for |r - r0| < R, r0 > R.

    V < E on the shell r0 - R t(E) < r < r0 + R t(E), t(E) = sqrt(1 - exp(-2E/(K R^2))), whose
    volume is (4 pi / 3)[(r0 + R t)^3 - (r0 - R t)^3]; a bin [E_a, E_b) holds the difference.
    """
    with mpmath.workdps(dps):
        KR2 = mpmath.mpf(K) * mpmath.mpf(R) ** 2
        r0m, Rm = mpmath.mpf(r0), mpmath.mpf(R)

        def vol(E):
            E = mpmath.mpf(E)
            if E <= 0:
                return mpmath.mpf(0)
            t = mpmath.sqrt(1 - mpmath.exp(-2 * E / KR2))
            return 4 * mpmath.pi / 3 * ((r0m + Rm * t) ** 3 - (r0m - Rm * t) ** 3)

        return [float(vol(b) - vol(a)) for a, b in zip(e_edges[:-1], e_edges[1:])]
