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
* ``fene_lj_trimer_omega``: binned density of states of three beads, two FENE
  bonds and the Lennard-Jones pair (0, 2), by a quadrature whose innermost
  integral is done in closed form (both parameter sets of Eq. (7)).
"""
from __future__ import annotations

import math

import mpmath
import numpy as np


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


def fene_lj_trimer_omega(e_edges, K: float, R: float, rc, n: int = 400, r0: float = 0.0,
                         sigma: float = 1.0):
    """Relative binned density of states of the N = 3 chain of Eq. (7): FENE bonds
    V_F(r) = -(K/2) R^2 ln(1 - ((r - r0)/R)^2) (|r - r0| < R) on (0, 1) and (1, 2), and the
    Lennard-Jones pair (0, 2), V_LJ(s) = 4 ((sigma/s)^12 - (sigma/s)^6) - V_c for s < rc, else 0,
    with V_c the unshifted value at rc (truncated and shifted; rc = None: no cutoff, V_c = 0).
    The benchmark configuration's reading is r0 = 0, R = 1.5, sigma = 1, rc = 2.5; the paper's own
    set is r0 = 0.7, R = 0.3, sigma = 2^(-1/6) r0, no cutoff.

    With bead 1 at the origin the bond vectors a = x0 - x1 and b = x2 - x1 are independent and
    uniform in the shell |r - r0| < R, and the (0, 2) distance is s = |a - b|.  In spherical
    coordinates d^3a d^3b = 8 pi^2 r_a^2 r_b^2 dr_a dr_b dc, c the cosine of the angle between a and
    b, and s^2 = r_a^2 + r_b^2 - 2 r_a r_b c turns dc into s ds / (r_a r_b).  So the volume with
    energy below E is

        C(E) = 8 pi^2 int int r_a r_b m(r_a, r_b) dr_a dr_b,
        m = int over s in [|r_a - r_b|, r_a + r_b] with V_LJ(s) < t of s ds,  t = E - V_F(r_a) - V_F(r_b).

    {s : V_LJ(s) < t} is an interval: with x = (sigma/s)^6, 4 (x^2 - x) = t + V_c has the roots
    x = (1 +- sqrt(1 + t + V_c)) / 2; the larger gives the inner end, the smaller the outer one
    for t <= 0 (for t > 0 the interval is unbounded: V_LJ < 0 up to rc and 0 beyond), and the set
    is empty below the well's bottom.  m is then (hi^2 - lo^2)/2 exactly; the outer double integral
    is a midpoint rule in w = sqrt(V_F) for each bond, n points on each side of r0 (the integrand
    is continuous and piecewise smooth), up to the top edge; the node spacing grows with that edge,
    so it suits windows of a few tens of energy units (n = 400 agrees with n = 1600 to ~4e-3 in
    the bins of the configuration's N = 3 window, ~1e-3 in the paper model's).  A bin [E_a, E_b)
    holds C(E_b) - C(E_a).
    """
    vc = 0.0 if rc is None else 4.0 * ((sigma / rc) ** 12 - (sigma / rc) ** 6)
    if not (r0 == 0.0 or r0 >= R):
        raise ValueError("the bond shell must not reach r = 0 unless r0 = 0")
    # One bond: nodes uniform in w = sqrt(V_F) (equal energy resolution up to the top of the window;
    # dr/dw stays finite at w = 0), on both sides of r0 when r0 > 0.  Bonds above
    # E_max - min V_LJ contribute to no bin.
    KR2 = K * R * R
    w_max = math.sqrt(max(e_edges[-1], 0.0) + 1.0 + abs(vc))
    dw = w_max / n
    w = (np.arange(n) + 0.5) * dw
    v = w * w
    q = np.exp(-2.0 * v / KR2)
    sv = np.sqrt(-np.expm1(-2.0 * v / KR2))
    drdw = 2.0 * w * R * q / (KR2 * sv) * dw
    r = np.concatenate([r0 + R * sv, r0 - R * sv]) if r0 > 0.0 else R * sv
    dr = np.concatenate([drdw, drdw]) if r0 > 0.0 else drdw
    vb = np.concatenate([v, v]) if r0 > 0.0 else v
    ia, ib = np.triu_indices(r.size)     # the integrand is symmetric in (r_a, r_b)
    ra, rb = r[ia], r[ib]
    wgt = np.where(ia != ib, 2.0, 1.0) * ra * rb * dr[ia] * dr[ib] * 8.0 * np.pi ** 2
    vf = vb[ia] + vb[ib]
    ra, rb = np.maximum(ra, rb), np.minimum(ra, rb)
    s_lo, s_hi = ra - rb, ra + rb

    def cum(E):
        t = E - vf
        disc = 1.0 + t + vc
        ok = disc > 0.0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        inner = sigma * ((1.0 + sq) / 2.0) ** (-1.0 / 6.0)
        xm = (1.0 - sq) / 2.0
        outer = np.where(t > 0.0, np.inf,
                         np.where(xm > 0.0, sigma * np.maximum(xm, 1e-300) ** (-1.0 / 6.0), np.inf))
        lo = np.maximum(s_lo, inner)
        hi = np.minimum(s_hi, outer)
        m = np.where(ok & (hi > lo), (hi * hi - lo * lo) / 2.0, 0.0)
        return float((wgt * m).sum())

    c = [cum(float(e)) for e in e_edges]
    return [b - a for a, b in zip(c[:-1], c[1:])]
