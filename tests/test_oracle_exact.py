"""Pins for the exact tools: brute force == transfer matrix == Kaufman's closed form,
plus the textbook invariants of Omega(E).  These tools in turn pin the MUCA oracle."""
import os

import mpmath
import numpy as np
import pytest

import oracle.exact as ex


def test_ising_bruteforce_equals_tm(orc):
    bf = [int(x) for x in orc.bruteforce_ising(4)]
    assert bf == orc.tm_ising(4)


@pytest.mark.parametrize("L", [4, 6, 8])
def test_ising_tm_equals_kaufman(orc, L):
    om = orc.tm_ising(L)
    N = L * L
    Es = [4 * j - 2 * N for j in range(N + 1)]
    for beta in (0.05, 0.3, float(mpmath.log(1 + mpmath.sqrt(2)) / 2), 0.6, 1.0):
        a = ex.lnZ_from_omega(om, Es, beta)
        b = ex.kaufman_lnZ(L, L, beta)
        assert abs(a - b) < mpmath.mpf(10) ** -40 * abs(b)


@pytest.fixture(scope="module")
def omega8(orc):
    return orc.tm_ising(8)


def test_ising_L8_invariants(omega8):
    N = 64
    om = omega8
    assert sum(om) == 2 ** N
    assert om == om[::-1]                     # Omega(E) = Omega(-E) for even L
    assert om[0] == 2 and om[1] == 0          # ground state doubly degenerate, no 2-bond state
    assert om[2] == 2 * N and om[3] == 4 * N  # one flipped spin; two neighbouring flipped spins


def test_ising_L8_golden_file(omega8):
    """tests/golden/ising_L8_omega.txt was written by tests/golden/make_golden.py (oracle only)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "ising_L8_omega.txt")
    vals = [int(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")]
    assert vals == omega8


@pytest.mark.parametrize("L", [4, 6, 8])
def test_ising_reachable_rule(orc, L, omega8):
    om = omega8 if L == 8 else orc.tm_ising(L)
    r = orc.Run(orc.ISING, L, 2, 1, 1)
    np.testing.assert_array_equal(r.reachable(), np.array(om) > 0)


def test_potts_bruteforce_equals_tm(orc):
    bf = [int(x) for x in orc.bruteforce_potts(4, 3)]
    assert bf == orc.tm_potts(4, 3)


@pytest.mark.parametrize("q,L", [(2, 4), (3, 4), (4, 4), (5, 4), (3, 6)])
def test_potts_invariants_and_reachable(orc, q, L):
    om = orc.tm_potts(L, q)
    N = L * L
    assert sum(om) == q ** N
    assert om[0] == q                          # E = -2N: all spins equal
    assert om[4] == (q * (q - 1) * N if q > 2 else 2 * N)  # one site differs from its 4 neighbours
    assert om[6] == q * (q - 1) * 2 * N                # a domino of one new colour (6 broken bonds)
    assert om[7] == q * (q - 1) * (q - 2) * 2 * N      # a domino of two new colours (7)
    r = orc.Run(orc.POTTS, L, q, 1, 1)
    np.testing.assert_array_equal(r.reachable(), np.array(om) > 0)


def test_potts_q2_is_ising(orc):
    """q = 2 Potts: E_P = -2N + n_b and E_I = -2N + 2 n_b, so Omega_P(n_b) = Omega_I(n_b / 2)."""
    L, N = 4, 16
    p = orc.tm_potts(L, 2)
    i = orc.tm_ising(L)
    for nb in range(2 * N + 1):
        assert p[nb] == (i[nb // 2] if nb % 2 == 0 else 0)


def test_ising_EM_bruteforce_equals_tm_and_marginals(orc):
    bf = orc.bruteforce_ising_EM(4)
    tm = orc.tm_ising_EM(4)
    assert [[int(x) for x in row] for row in bf] == tm
    tm6 = orc.tm_ising_EM(6)
    assert [sum(row) for row in tm6] == orc.tm_ising(6)
    for row in tm6:
        assert row == row[::-1]                # Omega(E, M) = Omega(E, -M)


@pytest.mark.parametrize("L", [16, 32])
def test_ising_kaufman_golden_files(L):
    """tests/golden/ising_L{16,32}_kaufman.txt (the GPU physics test, the configuration-2 run) are
    what their generator computes from Kaufman's closed form: ln Z at every beta, and <E>/N, C/N
    by central differences, re-derived here at beta = 0.4 with a different step."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ising_L%d_kaufman.txt" % L)
    rows = [[mpmath.mpf(x) for x in line.split()] for line in open(path) if not line.startswith("#")]
    assert len(rows) == 6
    for beta, lnZ, _, _ in rows:
        assert abs(ex.kaufman_lnZ(L, L, beta) - lnZ) < mpmath.mpf(10) ** -15 * abs(lnZ)
    beta, _, e, c = next(r for r in rows if abs(r[0] - mpmath.mpf("0.4")) < 1e-12)
    with mpmath.workdps(60):
        h = mpmath.mpf("1e-9")
        f = lambda t: ex.kaufman_lnZ(L, L, t)  # noqa: E731
        d1 = (f(beta + h) - f(beta - h)) / (2 * h)
        d2 = (f(beta + h) - 2 * f(beta) + f(beta - h)) / (h * h)
    assert abs(-d1 / (L * L) - e) < 1e-12
    assert abs(beta * beta * d2 / (L * L) - c) < 1e-8


def test_potts_q8_L4_golden_file(orc):
    """The stored 4x4 q = 8 Omega (written by tests/golden/make_golden.py from the oracle's transfer
    matrix): q^N states in all, the low-lying counts by hand (one site: q(q-1)N; a domino of one
    or two new colours: 2N q(q-1), 2N q(q-1)(q-2)) and the unreachable bins of the rule."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "potts_q8_L4_omega.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    E = [int(r[0]) for r in rows]
    om = [int(r[1]) for r in rows]
    q, N = 8, 16
    assert E == list(range(-2 * N, 1))
    assert sum(om) == q ** N
    assert om[0] == q and om[4] == q * (q - 1) * N
    assert om[6] == 2 * N * q * (q - 1) and om[7] == 2 * N * q * (q - 1) * (q - 2)
    assert [b for b in range(2 * N + 1) if om[b] == 0] == [1, 2, 3, 5]
    r = orc.Run(orc.POTTS, 4, q, 1, 1)
    np.testing.assert_array_equal(r.reachable(), np.array(om) > 0)



@pytest.mark.parametrize("model", [0, 1])
def test_trimer_quadrature_matches_direct_sampling(model):
    """The N = 3 quadrature (oracle/exact.py) against the definition sampled directly: 4e6 pairs of
    bond vectors drawn uniformly in the bond ball (model 0) or shell (model 1), their energy
    V_F(a) + V_F(b) + V_LJ(|a - b|) binned.  Every bin of the window within 4.5 standard
    deviations of the quadrature's share of the bond-pair volume, chi^2 per bin below 1.5."""
    K = 40.0
    if model == 0:
        R, r0, lo = 1.5, 0.0, 10.7
        kw = dict(K=K, R=R, rc=2.5)
    else:
        R, r0, lo = 0.3, 0.7, -0.9
        kw = dict(K=K, R=R, rc=None, r0=r0, sigma=2.0 ** (-1.0 / 6.0) * r0)
    edges = [lo + 0.1 * k for k in range(81)]
    r_in, r_out = max(r0 - R, 0.0), r0 + R
    vol = 4.0 * np.pi / 3.0 * (r_out ** 3 - r_in ** 3)
    rng = np.random.default_rng(5)
    n = 4_000_000

    def bonds():
        r = (r_in ** 3 + rng.random(n) * (r_out ** 3 - r_in ** 3)) ** (1.0 / 3.0)
        v = rng.normal(size=(n, 3))
        return r, v * (r / np.linalg.norm(v, axis=1))[:, None]

    ra, a = bonds()
    rb, b = bonds()
    vf = -(K * R * R / 2.0) * (np.log1p(-((ra - r0) / R) ** 2) + np.log1p(-((rb - r0) / R) ** 2))
    s = np.linalg.norm(a - b, axis=1)
    if model == 0:
        vl = np.where(s < 2.5, 4.0 * (s ** -12 - s ** -6) - 4.0 * (2.5 ** -12 - 2.5 ** -6), 0.0)
    else:
        sg = 2.0 ** (-1.0 / 6.0) * r0
        vl = 4.0 * ((sg / s) ** 12 - (sg / s) ** 6)
    h, _ = np.histogram(vf + vl, bins=np.array(edges))
    expect = np.array(ex.fene_lj_trimer_omega(edges, **kw)) / vol ** 2 * n
    z = (h - expect) / np.sqrt(expect)
    assert np.abs(z).max() < 4.5 and np.mean(z * z) < 1.5, (np.abs(z).max(), np.mean(z * z))


def test_oracle_muca_reproduces_kaufman_thermodynamics_L16(orc):
    """The whole oracle loop at 16x16 (beyond any enumeration here): 8 seeds of 64 walkers, 20
    iterations of 2000 sweeps, then Eq. 2 at the golden file's betas (Kaufman's closed form).
    <E>/N, C/N and ln Z (normalised at the ground state) each within 4 standard errors of the
    8-seed mean, plus 1e-4 of the value."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ising_L16_kaufman.txt")
    gold = [[float(x) for x in l.split()] for l in open(path) if l.strip() and not l.startswith("#")]
    N = 256
    vals = []
    for seed in range(1, 9):
        r = orc.Run(0, 16, 2, 64, seed)
        r.init()
        for _ in range(20):
            r.iterate(2000, 8)
            r.update()
        row = []
        for beta, _, _, _ in gold:
            out, _ = r.reweight(beta)
            row.append((out[0] / N, out[2], out[3]))
        vals.append(row)
    v = np.array(vals)                     # seeds x betas x (E/N, C/N, lnZ)
    mean = v.mean(axis=0)
    err = v.std(axis=0, ddof=1) / np.sqrt(v.shape[0])
    exact = np.array([[e, c, lz] for _, lz, e, c in gold])
    assert np.all(np.abs(mean - exact) < 4.0 * err + 1e-4 * np.abs(exact)), np.max(np.abs(mean - exact) / err)

