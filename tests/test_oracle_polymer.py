"""Pins for the polymer oracle (Eq. 7 reading): pair potentials against their defining
properties, exact energy bookkeeping, exact dyadic moves, and multicanonical sampling of the
FENE dimer against its closed-form binned density of states and of the FENE + LJ trimer against
its density of states by quadrature."""
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
    assert P.drift() < 1e-9            # the running sum matched the refresh after every call
    assert int(P.histogram().sum()) <= 8 * 200 * 13



def test_bin_width_and_cube_side_are_parameters(orc):
    """Bins of width 1/k and moves in a cube of side Q/4096: every walker's bin is
    floor((E - e_lo) k), and over one sweep every bead moves relative to bead 0 by whole grid steps
    Q 2^-44, at most the side Q 2^-12 per axis (bead and bead 0 each move at most half of it); a
    planted default step would move some bead by more than Q 2^-12."""
    lo, hi, Q = 33.3, 87.3, 300
    P = orc.PolyRun(13, 8, 5, lo, hi, bin_k=5, step_q=Q)
    assert P.B == round((hi - lo) * 5)
    P.init()
    P.iterate(300, 4)   # walk in
    P.update()
    X0 = P.coords().copy()
    P.iterate(1, 4)
    P.update()
    d = (P.coords() - X0) * 2.0 ** 44
    assert np.all(d % Q == 0) and np.abs(d).max() <= Q * 2.0 ** 32
    E, b = P.energy(), P.bins()
    inside = (E >= lo) & (E < hi)
    assert inside.any()
    np.testing.assert_array_equal(b[inside], np.floor((E[inside] - lo) * 5).astype(int))
    with pytest.raises(ValueError):
        orc.PolyRun(13, 8, 5, lo, hi, bin_k=0)


def test_walk_in_never_moves_away_and_records_inside_only(orc):
    """Thermalisation reading: random-walk chains start far above the N = 13 pilot window; outside
    it a move is accepted only if it does not increase the distance to the window, and only attempts
    made inside count.  Sweep by sweep: no walker's distance grows, a walker inside stays inside,
    and the iteration's histogram holds between N x (walkers inside at its start) and N x (walkers
    inside at its end) counts.  All 16 chains are in within 200 sweeps."""
    lo, hi, N, p = 33.3, 87.3, 13, 16
    P = orc.PolyRun(N, p, 3, lo, hi)
    P.init()

    def dist():
        E = P.energy()
        return np.maximum(np.maximum(E - hi, lo - E), 0.0)

    d = dist()
    assert np.all(d > 200.0)
    for _ in range(200):
        P.iterate(1, 4)
        P.update()
        d2 = dist()
        assert np.all(d2 <= d + 1e-9)
        assert np.all(d2[d == 0.0] == 0.0)
        n_in0, n_in1 = int((d == 0.0).sum()), int((d2 == 0.0).sum())
        assert N * n_in0 <= int(P.histogram().sum()) <= N * n_in1
        d = d2
        if np.all(d == 0.0):
            break
    assert np.all(d == 0.0)

@pytest.mark.parametrize("bin_k,step_q", [(10, 1229), (4, 819)])
def test_fene_dimer_density_of_states(orc, bin_k, step_q):
    """N = 2: the energy is the FENE energy of the bond vector, uniform in the ball r < R, so the
    binned density of states is (4 pi/3)(r(E_b)^3 - r(E_a)^3) with r(E) = R sqrt(1 - exp(-2E/(K R^2))).
    Also with bins of width 0.25 and moves in a cube of side 819/4096 = 0.2."""
    e_lo, e_hi = 0.0, 12.0
    P = orc.PolyRun(2, 64, 11, e_lo, e_hi, bin_k=bin_k, step_q=step_q)
    P.init()
    for _ in range(14):
        P.iterate(3000, 8)
        P.update()
    B = P.B
    assert B == round(12.0 * bin_k)
    edges = [e_lo + b / bin_k for b in range(B + 1)]
    omega = np.array(ex.fene_dimer_omega(edges, 40.0, 1.5))
    H = P.histogram().astype(float)
    seen = H > 0
    assert seen.mean() > 0.98
    lo = np.log(H[seen]) - P.lnW_sampled()[seen]
    le = np.log(omega[seen])
    off = np.median(le - lo)
    assert np.max(np.abs(lo + off - le)) < 0.15
    # Eq. 2 at bin centres: the oracle's reweighting equals the formula written out on its own
    # estimate ln H - ln W, and, from the exact binned Omega, <E> within the estimate's spread
    centres = np.array(edges[:-1]) + 0.5 / bin_k
    for beta in (0.5, 1.0):
        out, _ = P.reweight(beta)
        la = lo - beta * centres[seen]
        w = np.exp(la - la.max())
        e1 = float((w * centres[seen]).sum() / w.sum())
        e2 = float((w * centres[seen] ** 2).sum() / w.sum())
        assert abs(out[0] - e1) < 1e-9 * max(1.0, abs(e1))
        assert abs(out[1] - e2) < 1e-9 * max(1.0, abs(e2))
        assert abs(out[2] - beta * beta * (e2 - e1 * e1) / 2) < 1e-9 * max(1.0, out[2])
        lx = le - beta * centres[seen]
        wx = np.exp(lx - lx.max())
        ex_e = float((wx * centres[seen]).sum() / wx.sum())
        assert abs(out[0] - ex_e) < 0.02 * ex_e, (beta, out[0], ex_e)



@pytest.mark.parametrize("model,moves", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_fene_lj_trimer_density_of_states(orc, model, moves):
    """N = 3: two FENE bonds and the Lennard-Jones pair (0, 2), the smallest chain in which every
    term of Eq. (7) acts and a middle bead moves two bonds and the pair at once.  The oracle's
    multicanonical estimate ln H - ln W over a window from just above the lowest energy against
    the binned density of states by quadrature (inner integral in closed form), in the
    configuration's reading (model 0, lowest energy ~10.62) and with the paper's parameters
    (model 1, lowest energy -1: an equilateral triangle of side r0).  Mistakes this fails on:
    model 0, a wrong sign of the LJ shift (0.27 in some bin), a cutoff of 2 or 3, K = 41, R = 1.49;
    model 1, sigma = r0 (0.28), a cutoff at 2.5 sigma, R = 0.29.  The estimate's own deviation is
    ~0.01 rms.  With spherical rotations in the move set (moves = 1) the same Omega must come out:
    rotating an end bead about its neighbour changes only the LJ pair, the middle bead one bond
    and the pair."""
    if model == 0:
        e_lo, e_hi, sweeps, final = 10.7, 18.7, 12000, 0
        omega_args = dict(K=40.0, R=1.5, rc=RC)
    else:
        e_lo, e_hi, sweeps, final = -0.9, 7.1, 6000, 30000
        omega_args = dict(K=40.0, R=0.3, rc=None, r0=0.7, sigma=2.0 ** (-1.0 / 6.0) * 0.7)
    P = orc.PolyRun(3, 64, 13, e_lo, e_hi, model=model, moves=moves)
    P.init()
    for _ in range(14):
        P.iterate(sweeps, 8)
        P.update()
    if final:   # one long iteration on the converged weights (the thin top shells, as for N = 2)
        P.iterate(final, 8)
        P.update()
    B = P.B
    edges = [e_lo + 0.1 * b for b in range(B + 1)]
    omega = np.array(ex.fene_lj_trimer_omega(edges, **omega_args))
    assert omega.max() / omega.min() > 10
    H = P.histogram().astype(float)
    assert np.all(H > 0)
    lo = np.log(H) - P.lnW_sampled()
    le = np.log(omega)
    d = lo + np.median(le - lo) - le
    assert np.max(np.abs(d)) < 0.05 and np.sqrt(np.mean(d * d)) < 0.02
    # Eq. 2 at bin centres against the same sums over the exact binned Omega
    centres = np.array(edges[:-1]) + 0.05
    for beta in (0.5, 2.0):
        out, _ = P.reweight(beta)
        lx = le - beta * centres
        wx = np.exp(lx - lx.max())
        ex_e = float((wx * centres).sum() / wx.sum())
        assert abs(out[0] - ex_e) < 0.005 * max(1.0, abs(ex_e)), (beta, out[0], ex_e)


def test_paper_model_pair_potentials(orc):
    """Model 1 (Eq. 7 with K = 40, r0 = 0.7, r_max = 1): LJ zero at sigma = 2^(-1/6) r0 and
    minimum -1 at r0 with zero slope; FENE zero at r0, symmetric about it, (K/2) R^2 ln 2 at
    |r - r0| = R/sqrt(2), infinite at r0 +- R; no cutoff (LJ nonzero at r = 3)."""
    r0, R, K = 0.7, 0.3, 40.0
    sigma = 2.0 ** (-1.0 / 6.0) * r0
    assert abs(orc.poly_pair(sigma, 2, 1)) < 1e-13
    assert abs(orc.poly_pair(r0, 2, 1) + 1.0) < 1e-13
    h = 1e-6
    assert abs(orc.poly_pair(r0 + h, 2, 1) - orc.poly_pair(r0 - h, 2, 1)) < 1e-9
    assert orc.poly_pair(r0 * 1.01, 2, 1) > -1.0 and orc.poly_pair(r0 * 0.99, 2, 1) > -1.0
    assert orc.poly_pair(3.0, 2, 1) < 0.0
    assert abs(orc.poly_pair(r0, 1, 1)) < 1e-15
    d = R / math.sqrt(2.0)
    want = 0.5 * K * R * R * math.log(2.0)
    assert abs(orc.poly_pair(r0 + d, 1, 1) - want) < 1e-12
    assert abs(orc.poly_pair(r0 - d, 1, 1) - want) < 1e-12
    assert math.isinf(orc.poly_pair(r0 + R, 1, 1)) and math.isinf(orc.poly_pair(r0 - R, 1, 1))


def test_paper_model_straight_chain_energy(orc):
    """A straight chain with bonds r0: every bond contributes 0 and each pair at distance k r0
    (k >= 2) contributes 4[(sigma/(k r0))^12 - (sigma/(k r0))^6] = 4[(1/2) k^-12 - ... ]:
    with sigma^6 = r0^6 / 2 the pair term is 4[k^-12/4 - k^-6/2] = k^-12 - 2 k^-6."""
    N, r0 = 12, 0.7
    X = np.zeros((N, 3))
    X[:, 0] = r0 * np.arange(N)
    want = sum((N - k) * (k ** -12.0 - 2.0 * k ** -6.0) for k in range(2, N))
    assert abs(orc.poly_energy(X, 1) - want) < 1e-12


def test_paper_model_init_bonds(orc):
    """Initial chains of model 1: bonds of length r0 = 0.7 (to the grid rounding), no bead
    closer than 0.9 r0 to an earlier one, finite energy."""
    P = orc.PolyRun(40, 6, 5, -1e6, 1e6, model=1)
    P.init()
    X = P.coords()
    b = np.linalg.norm(np.diff(X, axis=1), axis=2)
    assert np.all(np.abs(b - 0.7) < 1e-12)
    for w in range(X.shape[0]):
        d = np.linalg.norm(X[w][:, None, :] - X[w][None, :, :], axis=2)
        iu = np.triu_indices(40, 2)
        assert d[iu].min() >= 0.63 - 1e-12
        assert abs(P.energy()[w] - orc.poly_energy(X[w], 1)) < 1e-9


def test_paper_model_dimer_density_of_states(orc):
    """N = 2 in model 1: the binned density of states of the shifted FENE bond against the closed
    form (4 pi/3)[(r0 + R t)^3 - (r0 - R t)^3], t = sqrt(1 - exp(-2E/(K R^2))).  The top bins are
    shells ~1e-3 thick that walkers enter rarely; with no thermalisation between iterations a
    3000-sweep iteration still carries the previous weights' distribution there (up to 0.1 in
    ln Omega), so the estimate comes from a final 30000-sweep iteration."""
    e_lo, e_hi = 0.0, 6.0
    P = orc.PolyRun(2, 64, 13, e_lo, e_hi, model=1)
    P.init()
    for _ in range(14):
        P.iterate(3000, 8)
        P.update()
    P.iterate(30000, 8)
    P.update()
    edges = [e_lo + 0.1 * b for b in range(P.B + 1)]
    omega = np.array(ex.fene_shifted_dimer_omega(edges, 40.0, 0.3, 0.7))
    H = P.histogram().astype(float)
    seen = H > 0
    assert seen.mean() > 0.98
    lo = np.log(H[seen]) - P.lnW_sampled()[seen]
    le = np.log(omega[seen])
    off = np.median(le - lo)
    # each bin within 4 counting errors (1/sqrt(H)) plus the error of the fitted offset
    assert np.all(np.abs(lo + off - le) < 4.0 / np.sqrt(H[seen]) + 0.03)


@pytest.mark.parametrize("model", [0, 1])
def test_rotation_moves_are_exact_and_energy_tracks(orc, model):
    """Move set 1 (shifts and spherical rotations): coordinates stay on the 2^-44 grid and the
    running energy equals the energy from scratch."""
    N = 40 if model == 1 else 13
    lo, hi = (-143.3, -4.2) if model == 1 else (33.3, 87.3)
    P = orc.PolyRun(N, 8, 9, lo, hi, model=model, moves=1)
    P.init()
    for _ in range(3):
        P.iterate(100, 8)
        P.update()
    X = P.coords()
    assert np.all(X * 2.0 ** 44 == np.round(X * 2.0 ** 44))
    E = P.energy()
    for w in range(8):
        assert E[w] == pytest.approx(orc.poly_energy(X[w], model), abs=1e-8)
    assert P.drift() < 1e-8


def test_rotation_directions_are_uniform(orc):
    """N = 2 at beta -> 0 with rotations: every rotation keeps the bond length and puts the bond
    on a uniform point of the sphere, so cos(theta) of the bond is uniform on [-1, 1] and its
    azimuth uniform on [-pi, pi) (a wrong Marsaglia formula would bias either)."""
    P = orc.PolyRun(2, 512, 21, -1e6, 1e6, beta=1e-12, moves=1)
    P.init()
    c, phi = [], []
    for _ in range(40):
        P.iterate(5, 8)
        X = P.coords()
        b = X[:, 1, :] - X[:, 0, :]
        c.extend((b[:, 2] / np.linalg.norm(b, axis=1)).tolist())
        phi.extend(np.arctan2(b[:, 1], b[:, 0]).tolist())
    c, phi = np.array(c), np.array(phi)
    hc, _ = np.histogram(c, bins=10, range=(-1, 1))
    hp, _ = np.histogram(phi, bins=10, range=(-np.pi, np.pi))
    for h in (hc, hp):
        e = h.sum() / 10
        assert ((h - e) ** 2 / e).sum() < 40  # 9 dof; samples are correlated, so a loose bound


def test_rotation_keeps_the_dimer_density_of_states(orc):
    """The shifted-FENE dimer (model 1) sampled with shifts and rotations reproduces the same
    closed-form density of states (rotations keep the bond length; shifts make it ergodic).
    Only half of the moves change the bond length here, so counts in the thin top shells are
    correlated over longer times than 1/sqrt(H) assumes: the bound is 0.1 in ln Omega (three
    seeds average to within 0.04 of the closed form in every bin)."""
    e_lo, e_hi = 0.0, 6.0
    P = orc.PolyRun(2, 64, 17, e_lo, e_hi, model=1, moves=1)
    P.init()
    for _ in range(14):
        P.iterate(3000, 8)
        P.update()
    P.iterate(30000, 8)
    P.update()
    edges = [e_lo + 0.1 * b for b in range(P.B + 1)]
    omega = np.array(ex.fene_shifted_dimer_omega(edges, 40.0, 0.3, 0.7))
    H = P.histogram().astype(float)
    seen = H > 0
    assert seen.mean() > 0.98
    lo = np.log(H[seen]) - P.lnW_sampled()[seen]
    le = np.log(omega[seen])
    off = np.median(le - lo)
    assert np.max(np.abs(lo + off - le)) < 0.1
