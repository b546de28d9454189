"""Pins for the oracle's MUCA / multimagnetic chains, merge, recursion, thresholds and
reweighting (Eq. 1-3, Fig. 1 scheme), against exact results and invariants."""
import math
import os

import mpmath
import numpy as np
import pytest

import oracle.exact as ex

NT = 8  # oracle threads


def energy_from_spins(spins, system):
    """From-scratch energy of each lattice, E = -sum over right and down bonds."""
    s = spins.astype(np.int64)
    rt = np.roll(s, -1, axis=2)
    dn = np.roll(s, -1, axis=1)
    if system == 1:
        return -((s == rt).sum(axis=(1, 2)) + (s == dn).sum(axis=(1, 2)))
    return -((s * rt).sum(axis=(1, 2)) + (s * dn).sum(axis=(1, 2)))


def bins_from_spins(spins, system):
    N = spins.shape[1] * spins.shape[2]
    if system == 0:
        return (energy_from_spins(spins, 0) + 2 * N) // 4
    if system == 1:
        return energy_from_spins(spins, 1) + 2 * N
    return (spins.astype(np.int64).sum(axis=(1, 2)) + N) // 2


@pytest.mark.parametrize("system,q", [(0, 2), (1, 3), (1, 8), (2, 2)])
def test_bins_track_lattices(orc, system, q):
    r = orc.Run(system, 8, q, 16, 99, beta=0.44)
    r.init()
    np.testing.assert_array_equal(r.bins(), bins_from_spins(r.spins(), system))
    for _ in range(3):
        r.iterate(50, NT)
        r.update()
        np.testing.assert_array_equal(r.bins(), bins_from_spins(r.spins(), system))
    assert r.sweep_counter() == 150


def test_init_spins_are_uniform(orc):
    r = orc.Run(1, 32, 8, 64, 5)
    r.init()
    counts = np.bincount(r.spins().ravel(), minlength=8)
    exp = counts.sum() / 8
    assert ((counts - exp) ** 2 / exp).sum() < 30  # 7 dof


def test_first_sweep_accepts_everything(orc):
    """ln W = 0 gives T = always on every reachable move, so one sequential sweep
    flips every spin once: the lattice becomes its negative (Ising)."""
    r = orc.Run(0, 8, 2, 8, 3)
    r.init()
    s0 = r.spins().copy()
    T = r.thresholds()
    reach = r.reachable()
    for b in range(r.B):
        for k in range(5):
            b2 = b + k - 2
            ok = reach[b] and 0 <= b2 < r.B and reach[b2]
            assert T[b, k] == (0xFFFFFFFF if ok else 0)
    r.iterate(1, 1)
    np.testing.assert_array_equal(r.spins(), -s0)



@pytest.mark.parametrize("q", [3, 8, 16])
def test_first_potts_sweep_applies_a_uniform_proposal_at_every_site(orc, q):
    """Potts proposal reading: with ln W = 0 every proposal is accepted, so after one sweep each
    site has moved by (new - old) mod q = 1 + mulhi(u, q - 1), never 0 and uniform over the q - 1
    other colours (chi^2 over 32768 sites below its 0.1 % point)."""
    r = orc.Run(orc.POTTS, 8, q, 512, 7)
    r.init()
    s0 = r.spins().astype(np.int64)
    r.iterate(1, NT)
    d = (r.spins().astype(np.int64) - s0) % q
    assert d.min() >= 1
    counts = np.bincount(d.ravel(), minlength=q)[1:]
    expect = d.size / (q - 1)
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    chi2_999 = {1: 10.83, 6: 22.46, 14: 36.12}[q - 2]   # 0.1 % points, q - 2 degrees of freedom
    assert chi2 < chi2_999, (q, chi2)

@pytest.mark.parametrize("record", [0, 1])
def test_histogram_totals(orc, record):
    r = orc.Run(0, 8, 2, 32, 4, record=record)
    r.init()
    r.iterate(30, NT)
    r.iterate(20, NT)
    r.update()
    per = 64 if record == 0 else 1
    assert int(r.histogram().sum()) == 32 * 50 * per


def test_merge_is_partition_independent(orc):
    """Any split of the walkers into groups gives the same merged histogram (a4)."""
    a = orc.Run(1, 8, 5, 24, 17)
    b = orc.Run(1, 8, 5, 24, 17)
    a.init(); b.init()
    a.iterate(40, 1); a.update()
    for w0, w1 in ((0, 5), (5, 6), (6, 24)):
        b.iterate_range(40, w0, w1, 3)
    b.advance(40); b.update()
    np.testing.assert_array_equal(a.histogram(), b.histogram())
    np.testing.assert_array_equal(a.lnW(), b.lnW())
    np.testing.assert_array_equal(a.spins(), b.spins())


@pytest.mark.parametrize("case", ["ising_L8", "potts_q8_L4"])
def test_recursion_ideal_histogram_gives_minus_ln_omega(orc, case):
    """Feeding H = Omega (sampled with W = 1) returns ln W = -ln Omega + const; a second
    histogram proportional to Omega*W is flat and leaves ln W unchanged.  Ising L = 8 has one
    unreachable bin between reachable neighbours, 4x4 q = 8 Potts the gaps {1, 2, 3} and {5}."""
    if case == "ising_L8":
        om_int = orc.tm_ising(8)
        r = orc.Run(0, 8, 2, 1, 1)
    else:
        om_int = [int(x) for x in _golden_omega("potts_q8_L4_omega.txt")]
        r = orc.Run(orc.POTTS, 4, 8, 1, 1)
    om = np.array([float(x) for x in om_int])
    r.init()
    reach = r.reachable()
    np.testing.assert_array_equal(reach, om > 0)
    r.set_open_histogram(np.array(om_int, dtype=np.uint64))
    r.update()
    lnW = r.lnW()
    target = -np.log(om[reach])
    d = lnW[reach] - target
    assert np.max(np.abs(d - d[0])) < 1e-12 * np.max(np.abs(target))
    assert np.all(np.isneginf(lnW[~reach]))
    H2 = np.zeros(r.B, dtype=np.uint64)
    H2[reach] = np.round(1e12 * np.exp(np.log(om[reach]) + lnW[reach] - (np.log(om[reach]) + lnW[reach]).max()))
    r.set_open_histogram(H2)
    r.update()
    assert np.max(np.abs(r.lnW()[reach] - lnW[reach])) < 1e-9


def test_first_update_is_plain_w_over_h(orc):
    """kappa = 1 on the first update: W^(1)(E) = W^(0)(E)/H^(0)(E) (the simple recursion)."""
    rng = np.random.default_rng(0)
    r = orc.Run(1, 4, 3, 1, 1)
    r.init()
    reach = r.reachable()
    H = np.zeros(r.B, dtype=np.uint64)
    H[reach] = rng.integers(1, 10**9, reach.sum())
    r.set_open_histogram(H)
    r.update()
    d = r.lnW()[reach] + np.log(H[reach].astype(float))
    assert np.ptp(d) < 1e-12 * 30


def test_plain_update_is_w_over_h_every_iteration(orc):
    """recursion = 1 (the paper's simple rule W(n+1) = W(n)/H(n), log form): after two updates
    ln W = -ln H1 - ln H2 up to the constant that puts ln W(r_0) at 0; an empty bin (H = 0 taken
    as 1) keeps its weight; unreachable bins stay at -inf."""
    rng = np.random.default_rng(3)
    r = orc.Run(0, 4, 2, 1, 1, recursion=1)
    r.init()
    reach = r.reachable()
    idx = np.nonzero(reach)[0]
    H1 = np.zeros(r.B, dtype=np.uint64); H1[idx] = rng.integers(1, 10**6, idx.size)
    H2 = np.zeros(r.B, dtype=np.uint64); H2[idx] = rng.integers(1, 10**6, idx.size)
    H2[idx[4]] = 0
    r.set_open_histogram(H1); r.update()
    r.set_open_histogram(H2); r.update()
    lh = np.log(H1[idx].astype(float)) + np.log(np.maximum(H2[idx], 1).astype(float))
    want = -(lh - lh[0])
    np.testing.assert_allclose(r.lnW()[idx], want, rtol=0, atol=1e-11)
    assert np.all(np.isneginf(r.lnW()[~reach]))
    assert r.lnW()[idx[0]] == 0.0


def test_plain_and_accumulated_updates_agree_on_the_first_update(orc):
    """With every reachable bin visited, the first accumulated-statistics update (kappa = 1)
    and the plain rule give the same weights (up to rounding order)."""
    rng = np.random.default_rng(4)
    H = None
    out = []
    for mode in (0, 1):
        r = orc.Run(1, 4, 3, 1, 1, recursion=mode)
        r.init()
        reach = r.reachable()
        if H is None:
            H = np.zeros(r.B, dtype=np.uint64)
            H[reach] = rng.integers(1, 10**9, reach.sum())
        r.set_open_histogram(H)
        r.update()
        out.append(r.lnW()[reach])
    np.testing.assert_allclose(out[0], out[1], rtol=0, atol=1e-10)


@pytest.mark.parametrize("case", ["ising_L4", "potts_q8_L4"])
def test_plain_update_reaches_the_fixed_point_of_an_ideal_histogram(orc, case):
    """If the histogram is exactly Omega(E) W(E) (ideal sampling), one plain update gives
    ln W = -ln Omega + const: the sign and the bookkeeping of the rule (exact Omega of the
    4x4 Ising lattice by brute force; of 4x4 q = 8 Potts from the golden file, whose unreachable
    bins sit between reachable ones)."""
    if case == "ising_L4":
        r = orc.Run(0, 4, 2, 1, 1, recursion=1)
        omega = orc.bruteforce_ising(4).astype(float)
        scale = 1000.0
    else:
        r = orc.Run(orc.POTTS, 4, 8, 1, 1, recursion=1)
        omega = _golden_omega("potts_q8_L4_omega.txt")
        scale = 1.0
    r.init()
    reach = r.reachable()
    H = np.zeros(r.B, dtype=np.uint64)
    H[reach] = (omega[reach] * scale).astype(np.uint64)  # W = 1 initially
    r.set_open_histogram(H)
    r.update()
    idx = np.nonzero(reach)[0]
    lo = np.log(omega[idx])
    np.testing.assert_allclose(r.lnW()[idx], -(lo - lo[0]), rtol=0, atol=1e-11)


def test_recursion_is_a_weighted_mean_of_naive_estimates(orc):
    """After two updates each neighbour ratio lnR is the g-weighted mean of the two naive
    estimates R^(n) + ln h0 - ln h1, with g = h0 h1/(h0+h1) (accumulated statistics)."""
    rng = np.random.default_rng(1)
    r = orc.Run(0, 4, 2, 1, 1)
    r.init()
    reach = np.nonzero(r.reachable())[0]
    H1 = np.zeros(r.B, dtype=np.uint64); H1[reach] = rng.integers(1, 1000, reach.size)
    H2 = np.zeros(r.B, dtype=np.uint64); H2[reach] = rng.integers(1, 1000, reach.size)
    H2[reach[3]] = 0  # pairs touching an empty bin keep their ratio
    r.set_open_histogram(H1); r.update(); w1 = r.lnW()[reach]
    r.set_open_histogram(H2); r.update(); w2 = r.lnW()[reach]
    R1, R2 = np.diff(w1), np.diff(w2)
    for k in range(reach.size - 1):
        a1, c1 = float(H1[reach[k]]), float(H1[reach[k + 1]])
        a2, c2 = float(H2[reach[k]]), float(H2[reach[k + 1]])
        est1 = math.log(a1) - math.log(c1)       # naive estimate from W^(0) = 1
        if a2 == 0 or c2 == 0:
            assert R2[k] == pytest.approx(R1[k], abs=1e-12)
            continue
        est2 = R1[k] + math.log(a2) - math.log(c2)
        g1, g2 = a1 * c1 / (a1 + c1), a2 * c2 / (a2 + c2)
        assert R2[k] == pytest.approx((g1 * est1 + g2 * est2) / (g1 + g2), abs=1e-11)


def test_thresholds_match_exact_exponential(orc):
    rng = np.random.default_rng(2)
    r = orc.Run(1, 4, 3, 1, 1)
    r.init()
    reach = r.reachable()
    H = np.zeros(r.B, dtype=np.uint64)
    H[reach] = rng.integers(1, 10**6, reach.sum())
    r.set_open_histogram(H)
    r.update()
    lnW, T = r.lnW(), r.thresholds()
    n_exact = n = 0
    for b in np.nonzero(reach)[0]:
        for k in range(9):
            b2 = b + k - 4
            if not (0 <= b2 < r.B and reach[b2]):
                assert T[b, k] == 0
                continue
            d = lnW[b2] - lnW[b]
            if d >= 0:
                assert T[b, k] == 0xFFFFFFFF
                continue
            ref = int(mpmath.floor(mpmath.ldexp(mpmath.exp(mpmath.mpf(d)), 32)))
            assert abs(int(T[b, k]) - ref) <= 1
            n += 1
            n_exact += int(T[b, k]) == ref
    assert n > 50 and n_exact >= n - 1


def test_multimagnetic_thresholds_include_beta(orc):
    """MUMA (Eq. 3): d = ln W(M') - ln W(M) - beta dE; with ln W = 0 only beta dE remains."""
    beta = 0.4407
    r = orc.Run(2, 4, 2, 1, 1, beta=beta)
    r.init()
    T = r.thresholds()
    for b in range(1, r.B - 1):
        for sidx in range(2):
            for k in range(5):
                dE = 4 * (k - 2)
                t = T[b, sidx * 5 + k]
                if dE <= 0:
                    assert t == 0xFFFFFFFF
                else:
                    ref = int(mpmath.floor(mpmath.ldexp(mpmath.exp(-beta * dE), 32)))
                    assert abs(int(t) - ref) <= 1


def test_reweight_exact_omega(orc):
    """Eq. (2) on an exact histogram (H = Omega, W = 1) reproduces <E>, C_V and ln Z of
    direct summation and of Kaufman's formula."""
    om = orc.tm_ising(8)
    r = orc.Run(0, 8, 2, 1, 1)
    r.init()
    r.set_open_histogram(np.array(om, dtype=np.uint64))
    r.update()
    N = 64
    Es = [4 * j - 2 * N for j in range(N + 1)]
    for beta in (0.2, 0.4406868, 0.7):
        out, lnP = r.reweight(beta)
        with mpmath.workdps(50):
            b = mpmath.mpf(beta)
            w = [mpmath.mpf(o) * mpmath.exp(-b * E) for o, E in zip(om, Es)]
            Z = mpmath.fsum(w)
            e1 = mpmath.fsum(wi * E for wi, E in zip(w, Es)) / Z
            e2 = mpmath.fsum(wi * E * E for wi, E in zip(w, Es)) / Z
        assert out[0] == pytest.approx(float(e1), rel=1e-12, abs=1e-10)
        assert out[1] == pytest.approx(float(e2), rel=1e-12)
        assert out[2] == pytest.approx(float(b * b * (e2 - e1 * e1) / N), rel=1e-9)
        assert out[3] == pytest.approx(float(ex.kaufman_lnZ(8, 8, beta)), rel=1e-12)
        assert np.exp(lnP[np.isfinite(lnP)]).sum() == pytest.approx(1.0, rel=1e-12)



def test_reweight_exact_potts_q8_omega(orc):
    """Eq. (2) for the Potts model on an exact histogram (H = the golden 4x4 q = 8 Omega, W = 1):
    <E>, <E^2>, C_V per site and ln Z (ground state normalised to q states) equal direct summation
    at 50 digits, across the first-order transition (beta_c = ln(1 + sqrt 8) = 1.342)."""
    om = _golden_omega("potts_q8_L4_omega.txt")
    r = orc.Run(orc.POTTS, 4, 8, 1, 1)
    r.init()
    r.set_open_histogram(om.astype(np.uint64))
    r.update()
    N = 16
    Es = [b - 2 * N for b in range(2 * N + 1)]
    for beta in (0.5, 1.342, 2.5):
        out, lnP = r.reweight(beta)
        with mpmath.workdps(50):
            b = mpmath.mpf(beta)
            w = [mpmath.mpf(int(o)) * mpmath.exp(-b * E) for o, E in zip(om, Es)]
            Z = mpmath.fsum(w)
            e1 = mpmath.fsum(wi * E for wi, E in zip(w, Es)) / Z
            e2 = mpmath.fsum(wi * E * E for wi, E in zip(w, Es)) / Z
        assert out[0] == pytest.approx(float(e1), rel=1e-12)
        assert out[1] == pytest.approx(float(e2), rel=1e-12)
        assert out[2] == pytest.approx(float(b * b * (e2 - e1 * e1) / N), rel=1e-9)
        assert out[3] == pytest.approx(float(mpmath.log(Z)), rel=1e-12)
        assert np.exp(lnP[np.isfinite(lnP)]).sum() == pytest.approx(1.0, rel=1e-12)


def test_reweight_exact_multimagnetic_histogram(orc):
    """MUMA reweighting (reading of Eq. 2 over M at the run's own beta) on an exact histogram:
    H(M) = P_beta(M) (from the exact Omega(E, M) of 6x6, scaled to 1e15 and rounded) and W = 1 give
    <|M|>/N, <M^2>/N^2, the susceptibility beta N (<M^2>/N^2 - <|M|>^2/N^2) and
    ln P(M = 0) - ln P(M = N) of direct summation."""
    beta, L, N = 0.4407, 6, 36
    em = orc.tm_ising_EM(L)
    with mpmath.workdps(50):
        P = [mpmath.fsum(mpmath.mpf(em[j][m]) * mpmath.exp(-mpmath.mpf(beta) * (4 * j - 2 * N))
                         for j in range(N + 1)) for m in range(N + 1)]
        top = max(P)
        H = [int(mpmath.nint(mpmath.mpf(10) ** 15 * x / top)) for x in P]
        Hm = [mpmath.mpf(h) for h in H]
        Z = mpmath.fsum(Hm)
        absM = [abs(2 * m - N) for m in range(N + 1)]
        a1 = mpmath.fsum(h * a for h, a in zip(Hm, absM)) / Z / N
        a2 = mpmath.fsum(h * a * a for h, a in zip(Hm, absM)) / Z / N ** 2
        barrier = mpmath.log(Hm[N // 2]) - mpmath.log(Hm[N])
    r = orc.Run(2, L, 2, 1, 1, beta=beta)
    r.init()
    r.set_open_histogram(np.array(H, dtype=np.uint64))
    r.update()
    out, _ = r.reweight(beta)
    assert out[0] == pytest.approx(float(a1), rel=1e-12)
    assert out[1] == pytest.approx(float(a2), rel=1e-12)
    assert out[2] == pytest.approx(float(beta * N * (a2 - a1 * a1)), rel=1e-9)
    assert out[3] == pytest.approx(float(barrier), rel=1e-12)

def test_muca_converges_to_exact_ising_L8(orc):
    """The config-1 workload (L = 8, p = 64, 10 iterations of 1e4 sweeps): flat histogram and
    ln Omega_hat = ln H - ln W within 0.15 of Beale's exact Omega in every reachable bin."""
    om = np.array([float(x) for x in orc.tm_ising(8)])
    r = orc.Run(0, 8, 2, 64, 1)
    r.init()
    for _ in range(10):
        r.iterate(10000, NT)
        r.update()
    flat, st = r.is_flat(0.5)
    assert flat
    reach = r.reachable()
    lo = np.log(r.histogram()[reach].astype(float)) - r.lnW_sampled()[reach]
    le = np.log(om[reach])
    lo += le[0] - lo[0]   # normalise at the ground state, Omega(-2N) = 2
    assert np.max(np.abs(lo - le)) < 0.15



def test_muca_ising_L8_is_unbiased_over_16_seeds(orc):
    """The same workload from 16 seeds: in every reachable bin the mean deviation of ln Omega_hat
    (normalised at the ground state) from Beale's exact Omega lies within 4 standard errors of
    the 16-seed mean (for independent seeds the jackknife error of the mean) plus 0.005.  Single
    seeds reach 0.15; acceptance thresholds planted 0.2 % low in the oracle pass the single-run
    test above and fail this one."""
    om = np.array([float(x) for x in orc.tm_ising(8)])
    devs = []
    for seed in range(1, 17):
        r = orc.Run(0, 8, 2, 64, seed)
        r.init()
        for _ in range(10):
            r.iterate(10000, NT)
            r.update()
        reach = r.reachable()
        lo = np.log(r.histogram()[reach].astype(float)) - r.lnW_sampled()[reach]
        le = np.log(om[reach])
        devs.append(lo + (le[0] - lo[0]) - le)
    d = np.array(devs)[:, 1:]            # bin 0 is the normalisation
    mean = d.mean(axis=0)
    se = d.std(axis=0, ddof=1) / np.sqrt(d.shape[0])
    assert np.all(np.abs(mean) < 4.0 * se + 0.005), np.max(np.abs(mean) / se)
    assert se.max() < 0.02


def test_statistical_speedup_is_at_least_linear_for_ising_L8(orc):
    """Eq. 6 on the oracle: 16 seeds per p start from ln W = 0 with M(p) = round(5.7 L^2.51 / p)
    sweeps a walker per iteration (Eq. 4, the paper's Ising fit) and stop at their first flat merged
    histogram; S*_p = [N_iter M]_1 / [N_iter M]_p.  The paper finds S*_p close to p for the 2D Ising
    model up to p = 64 (Fig. 3); at L = 8 the oracle's S*_p is at least 0.9 p."""
    L = 8

    def m_opt(p):
        return max(1, int(round(5.7 * L ** 2.51 / p)))

    cost = {}
    for p in (1, 4, 16, 64):
        n = []
        for k in range(16):
            r = orc.Run(0, L, 2, p, 1000 + 7919 * k + p)
            r.init()
            for it in range(1, 501):
                r.iterate(m_opt(p), NT)
                r.update()
                if r.is_flat(0.5)[0]:
                    n.append(it)
                    break
        assert len(n) == 16, p
        cost[p] = float(np.mean(n)) * m_opt(p)
    for p in (4, 16, 64):
        assert cost[1] / cost[p] >= 0.9 * p, (p, cost[1] / cost[p])

def test_muca_potts_q3_L6_converges(orc):
    om = np.array([float(x) for x in orc.tm_potts(6, 3)])
    r = orc.Run(1, 6, 3, 64, 2)
    r.init()
    for _ in range(12):
        r.iterate(4000, NT)
        r.update()
    reach = r.reachable()
    lo = np.log(r.histogram()[reach].astype(float)) - r.lnW_sampled()[reach]
    le = np.log(om[reach])
    lo += le[0] - lo[0]
    assert np.max(np.abs(lo - le)) < 0.25



def _golden_omega(name):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    return np.array([float(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")])


def test_muca_potts_q8_L4_is_unbiased_over_16_seeds(orc):
    """q = 8 (the benchmark's q; proposals draw one of q - 1 = 7 colours, not a power of two) on
    the 4x4 torus: ln H - ln W against the exact Omega (golden file), which spans 28 units of
    ln Omega over 29 reachable bins.  Every seed within 0.2 in every bin; the 16-seed mean within
    4 standard errors + 0.005 per bin."""
    om = _golden_omega("potts_q8_L4_omega.txt")
    devs = []
    for seed in range(1, 17):
        r = orc.Run(orc.POTTS, 4, 8, 64, seed)
        r.init()
        for _ in range(12):
            r.iterate(4000, NT)
            r.update()
        reach = r.reachable()
        np.testing.assert_array_equal(reach, om > 0)
        lo = np.log(r.histogram()[reach].astype(float)) - r.lnW_sampled()[reach]
        le = np.log(om[reach])
        devs.append(lo + (le[0] - lo[0]) - le)
    d = np.array(devs)[:, 1:]
    assert np.abs(d).max() < 0.2
    mean = d.mean(axis=0)
    se = d.std(axis=0, ddof=1) / np.sqrt(d.shape[0])
    assert np.all(np.abs(mean) < 4.0 * se + 0.005), np.max(np.abs(mean) / se)

def test_multimagnetic_converges_to_exact_P_of_M(orc):
    """MUMA at beta = 0.4407, L = 6: ln W(M) -> -ln P_beta(M) + const, with
    P_beta(M) = sum_E Omega(E, M) exp(-beta E) from the exact transfer matrix."""
    beta, L, N = 0.4407, 6, 36
    em = orc.tm_ising_EM(L)
    with mpmath.workdps(40):
        lnPM = []
        for m in range(N + 1):
            s = mpmath.fsum(mpmath.mpf(em[j][m]) * mpmath.exp(-beta * (4 * j - 2 * N)) for j in range(N + 1))
            lnPM.append(float(mpmath.log(s)))
    lnPM = np.array(lnPM)
    r = orc.Run(2, L, 2, 64, 3, beta=beta)
    r.init()
    for _ in range(10):
        r.iterate(3000, NT)
        r.update()
    lo = np.log(r.histogram().astype(float)) - r.lnW_sampled()
    lo += lnPM[0] - lo[0]
    assert np.max(np.abs(lo - lnPM)) < 0.15
    out, _ = r.reweight(beta)
    with mpmath.workdps(30):
        P = np.exp(lnPM - lnPM.max()); P /= P.sum()
    absM = np.abs(2 * np.arange(N + 1) - N)
    assert out[0] == pytest.approx((P * absM).sum() / N, rel=0.02)



def test_multimagnetic_is_unbiased_over_16_seeds(orc):
    """The multimagnetic workload above from 16 seeds: every seed within 0.15 of -ln P_beta(M) in
    every bin, and the 16-seed mean within 4 standard errors + 0.005 per bin."""
    beta, L, N = 0.4407, 6, 36
    em = orc.tm_ising_EM(L)
    with mpmath.workdps(40):
        lnPM = np.array([float(mpmath.log(mpmath.fsum(mpmath.mpf(em[j][m]) * mpmath.exp(-beta * (4 * j - 2 * N))
                                                      for j in range(N + 1)))) for m in range(N + 1)])
    devs = []
    for seed in range(1, 17):
        r = orc.Run(2, L, 2, 64, seed, beta=beta)
        r.init()
        for _ in range(10):
            r.iterate(3000, NT)
            r.update()
        lo = np.log(r.histogram().astype(float)) - r.lnW_sampled()
        devs.append(lo + (lnPM[0] - lo[0]) - lnPM)
    d = np.array(devs)[:, 1:]
    assert np.abs(d).max() < 0.15
    mean = d.mean(axis=0)
    se = d.std(axis=0, ddof=1) / np.sqrt(d.shape[0])
    assert np.all(np.abs(mean) < 4.0 * se + 0.005), np.max(np.abs(mean) / se)

def _canonical_m_moments(orc, L, beta):
    """Exact <|M|>/N and <M^2>/N^2 at beta from the brute-force Omega(E, M)."""
    om = orc.bruteforce_ising_EM(L).astype(float)
    N = L * L
    E = 4.0 * np.arange(N + 1) - 2 * N
    M = 2.0 * np.arange(N + 1) - N
    w = om * np.exp(-beta * (E - E.min()))[:, None]
    z = w.sum()
    return (w * np.abs(M)[None, :]).sum() / z / N, (w * (M ** 2)[None, :]).sum() / z / N ** 2


@pytest.mark.parametrize("beta", [0.0, 0.3, 0.4407, 0.8])
def test_observable_reweighting_is_eq2(orc, beta):
    """Eq. 2 on per-bin sums: with sums that are exact expectations under any weights W
    (n(b) = c W(b) Omega(b), S_|M|(b) = c W(b) sum_M Omega(b, M)|M|, ...), the reweighted moments
    equal the exact canonical ones of the 4x4 Ising lattice."""
    L, N = 4, 16
    om = orc.bruteforce_ising_EM(L).astype(float)
    M = 2.0 * np.arange(N + 1) - N
    rng = np.random.default_rng(5)
    lnW = rng.uniform(-3, 3, N + 1)
    scale = 2.0 ** 20
    sums = np.zeros((N + 1, 3), dtype=np.uint64)
    # integer sums need the factor c e^{lnW} Omega to be integral: choose W so that it is
    for b in range(N + 1):
        if om[b].sum() == 0:
            continue
        f = np.round(scale * np.exp(lnW[b]))
        lnW[b] = np.log(f / scale)
        sums[b] = [f * om[b].sum(), f * (om[b] * np.abs(M)).sum(), f * (om[b] * M ** 2).sum()]
    got = orc.reweight_obs(N, sums, lnW, beta)
    m1, m2 = _canonical_m_moments(orc, L, beta)
    assert abs(got[0] - m1) < 1e-12 and abs(got[1] - m2) < 1e-12
    assert abs(got[2] - beta * N * (m2 - m1 ** 2)) < 1e-10


def test_observable_sums_follow_the_lattices(orc):
    """Per-sweep sums (reading R9): over one sweep of p walkers the sample count is p, and
    after the sweep the sums equal |M| and M^2 of the final lattices in their final bins."""
    r = orc.Run(0, 8, 2, 12, 7, observables=1)
    r.init()
    r.iterate(1, 1)
    r.update()
    S = r.observable_sums()
    s = r.spins().astype(np.int64)
    Mw = s.sum(axis=(1, 2))
    want = np.zeros(S.shape, dtype=np.int64)
    for w, b in enumerate(r.bins()):
        want[b] += np.array([1, abs(Mw[w]), Mw[w] ** 2], dtype=np.int64)
    np.testing.assert_array_equal(S.astype(np.int64), want)


def test_observables_at_low_temperature_from_a_muca_run(orc):
    """A short multicanonical run of the 4x4 Ising lattice: the reweighted <|M|>/N at
    beta = 0.6 is within 3% of the exact value (statistical check of the whole chain)."""
    r = orc.Run(0, 4, 2, 64, 11, observables=1)
    r.init()
    for _ in range(12):
        r.iterate(400, NT)
        r.update()
    got = r.reweight_observables(0.6)
    m1, _ = _canonical_m_moments(orc, 4, 0.6)
    assert abs(got[0] - m1) < 0.03 * m1


def test_flatness_is_min_over_mean_on_reachable_bins(orc):
    """Reading 9 written out: {min, mean, max} of the last merged histogram over the reachable
    bins, and flat iff every reachable bin is visited and min >= ratio * mean."""
    r = orc.Run(1, 6, 3, 16, 4)
    r.init()
    for it in range(6):
        r.iterate(300, 4)
        r.update()
        H = r.histogram()[r.reachable()].astype(float)
        for ratio in (0.2, 0.5, 0.8):
            flat, st = r.is_flat(ratio)
            assert st[0] == H.min() and st[2] == H.max()
            assert abs(st[1] - H.mean()) <= 1e-12 * H.mean()
            assert flat == bool(H.min() > 0 and H.min() >= ratio * H.mean())


@pytest.mark.parametrize("system,q,beta", [(0, 2, 0.3), (1, 3, 0.6)])
def test_fixed_canonical_weights_sample_the_canonical_ensemble(orc, system, q, beta):
    """ln W(E) = -beta E turns the multicanonical acceptance min(1, W(E')/W(E)) (Eq. 1) into
    Metropolis at beta: a run at these fixed weights samples exp(-beta E) Omega(E) / Z, with
    Omega(E) from brute-force enumeration of the 4x4 lattice.  Mean and variance of E over 16
    independent seeds agree with the exact values within 5 standard errors; lnW = 0 (every move
    accepted) or the opposite sign would miss both by many."""
    L, p, N = 4, 32, 16
    om = orc.bruteforce_ising(L) if system == 0 else orc.bruteforce_potts(L, q)
    Es = np.array([4 * b - 2 * N for b in range(N + 1)] if system == 0 else [b - 2 * N for b in range(2 * N + 1)],
                  dtype=np.float64)
    w = om.astype(np.float64) * np.exp(-beta * (Es - Es.min()))
    P = w / w.sum()
    e1, e2 = (P * Es).sum(), (P * Es * Es).sum()
    m1, m2 = [], []
    for seed in range(16):
        r = orc.Run(system, L, q, p, 500 + seed)
        r.init()
        for sweeps in (200, 2000):  # burn-in, then measurement
            r.set_lnW(-beta * Es)
            r.iterate(sweeps, NT)
            r.update()
        H = r.histogram().astype(np.float64)
        assert H.sum() == p * 2000 * N
        m1.append((H * Es).sum() / H.sum())
        m2.append((H * Es * Es).sum() / H.sum())
    for m, exact in ((np.array(m1), e1), (np.array(m2), e2)):
        se = m.std(ddof=1) / np.sqrt(m.size)
        assert abs(m.mean() - exact) < 5 * se + 1e-12, (m.mean(), exact, se)
    r = orc.Run(system, L, q, p, 1)
    r.init()
    r.set_lnW(-beta * Es)
    T = r.thresholds().reshape(r.B, r.K)
    reach = r.reachable().astype(bool)
    assert (T[~reach] == 0).all()
