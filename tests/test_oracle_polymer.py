"""Pins for the polymer oracle (Eq. 7 reading): pair potentials against their defining
properties, exact energy bookkeeping, exact dyadic moves, and multicanonical sampling of the
FENE dimer against its closed-form binned density of states."""
import math

import numpy as np
import pytest

import oracle.exact as ex

RC = 2.5


def test_lj_properties(orc):
    vrc = 4 * (RC ** -12 - RC ** -6)
    rmin = 2 ** (1 / 6)
    assert orc.poly_pair(RC, 2) == 0.0 and orc.poly_pair(3.0, 5) == 0.0       # truncated at the cutoff
    assert orc.poly_pair(RC - 1e-9, 2) == pytest.approx(0.0, abs=1e-7)       # ... and shifted: continuous
    assert orc.poly_pair(1.0, 2) == pytest.approx(-vrc, abs=1e-15)           # sigma = 1: LJ(1) = 0 before the shift
    assert orc.poly_pair(rmin, 3) == pytest.approx(-1.0 - vrc, rel=1e-14)    # well depth eps = 1 at 2^(1/6)
    h = 1e-6                                                                 # minimum at 2^(1/6)
    assert (orc.poly_pair(rmin + h, 2) - orc.poly_pair(rmin - h, 2)) / (2 * h) == pytest.approx(0.0, abs=1e-7)


def test_fene_properties(orc):
    K, R = 40.0, 1.5
    assert orc.poly_pair(0.0, 1) == 0.0
    r = 1e-4
    assert orc.poly_pair(r, 1) == pytest.approx(0.5 * K * r * r, rel=1e-6)  # harmonic limit
    assert math.isinf(orc.poly_pair(R, 1)) and math.isinf(orc.poly_pair(2.0, 1))
    r = 1.0   # exp(-2V/(K R^2)) = 1 - (r/R)^2
    assert math.exp(-2 * orc.poly_pair(r, 1) / (K * R * R)) == pytest.approx(1 - (r / R) ** 2, rel=1e-13)


def test_init_chain_geometry(orc):
    P = orc.PolyRun(32, 6, 5, 53.0, 176.7)
    P.init()
    X = P.coords()
    bond = np.linalg.norm(np.diff(X, axis=1), axis=2)
    assert np.all(np.abs(bond - 1.0) < 1e-12)
    for w in range(6):
        d = np.linalg.norm(X[w][:, None, :] - X[w][None, :, :], axis=2)
        iu = np.triu_indices(32, 2)
        assert (d[iu] >= 0.9 - 1e-12).mean() > 0.999
    # coordinates lie on the 2^-44 grid
    assert np.all(X * 2.0 ** 44 == np.round(X * 2.0 ** 44))
    E = P.energy()
    for w in range(6):
        assert E[w] == pytest.approx(orc.poly_energy(X[w]), rel=1e-14)


def test_moves_are_exact_and_energy_tracks(orc):
    P = orc.PolyRun(13, 8, 7, 33.3, 87.3)
    P.init()
    for _ in range(3):
        P.iterate(200, 8)
        P.update()
    X = P.coords()
    assert np.all(X * 2.0 ** 44 == np.round(X * 2.0 ** 44))   # still on the grid
    assert np.all(X[:, 0, :] == 0.0)                           # recentred on bead 0
    E = P.energy()
    for w in range(8):
        assert E[w] == pytest.approx(orc.poly_energy(X[w]), abs=1e-9)
    assert P.refresh_energy() < 1e-9
    assert int(P.histogram().sum()) <= 8 * 200 * 13


def test_fene_dimer_density_of_states(orc):
    """N = 2: the energy is the FENE energy of the bond vector, uniform in the ball r < R, so the
    binned density of states is (4 pi/3)(r(E_b)^3 - r(E_a)^3) with r(E) = R sqrt(1 - exp(-2E/(K R^2)))."""
    e_lo, e_hi = 0.0, 12.0
    P = orc.PolyRun(2, 64, 11, e_lo, e_hi)
    P.init()
    for _ in range(14):
        P.iterate(3000, 8)
        P.update()
    B = P.B
    edges = [e_lo + 0.1 * b for b in range(B + 1)]
    omega = np.array(ex.fene_dimer_omega(edges, 40.0, 1.5))
    H = P.histogram().astype(float)
    seen = H > 0
    assert seen.mean() > 0.98
    lo = np.log(H[seen]) - P.lnW_sampled()[seen]
    le = np.log(omega[seen])
    off = np.median(le - lo)
    assert np.max(np.abs(lo + off - le)) < 0.15
