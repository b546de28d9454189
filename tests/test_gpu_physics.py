"""The whole GPU path against exact physics at a size no enumeration reaches: eight independent
multicanonical runs of the 16x16 Ising model (512 walkers each, batched) iterate to a flat
histogram, refine with eight longer iterations, and reweight (Eq. 2) to six temperatures.  The
mean over the runs of <E>/N, C/N and ln Z must agree with Kaufman's exact finite-lattice values
(tests/golden/ising_L16_kaufman.txt, written by tests/golden/make_golden.py from oracle/exact.py)
within four standard errors of that mean.  The seeds are fixed, so the run is reproducible."""
import math
import os

import numpy as np
import pytest

import paper_1312_2213_gb300 as m

pytestmark = pytest.mark.gpu
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "ising_L16_kaufman.txt")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_ising_L16_thermodynamics_match_kaufman():
    gold = [tuple(float(x) for x in line.split()) for line in open(GOLD) if not line.startswith("#")]
    N = 256
    systems = [m.Muca(m.ISING2D, 16, 2, 512, s) for s in range(101, 109)]
    b = m.Batch(systems)
    for it in range(400):
        b.run(1, 20, use_graph=False)
        flat = [s.flatness() for s in systems]
        if all(f[0] > 0 and f[0] >= 0.5 * f[1] for f in flat):
            break
    else:
        pytest.fail("no flat histogram within 400 iterations")
    b.run(8, 500, use_graph=False)
    for beta, lnZ, e, c in gold:
        outs = np.array([s.reweight(beta)[0] for s in systems])  # {<E>, <E^2>, C/N, ln Z}
        for name, est, exact in (("E/N", outs[:, 0] / N, e), ("C/N", outs[:, 2], c), ("lnZ", outs[:, 3], lnZ)):
            mean, err = est.mean(), est.std(ddof=1) / math.sqrt(len(est))
            assert abs(mean - exact) < 4 * err, (beta, name, mean, exact, err)
    b.close()


def test_potts_q2_L16_maps_onto_kaufman():
    """q = 2 Potts is Ising with E_Potts = -N + E_Ising / 2: at beta_Potts = 2 beta the exact values
    are <E>/N = -1 + <E_Ising>/(2N), the same C/N, and ln Z = 2 beta N + ln Z_Ising.  The Potts
    code path (nibble lattices, its own producers and consumer) against them."""
    gold = [tuple(float(x) for x in line.split()) for line in open(GOLD) if not line.startswith("#")]
    N = 256
    systems = [m.Muca(m.POTTS2D, 16, 2, 512, s) for s in range(201, 209)]
    b = m.Batch(systems)
    for it in range(400):
        b.run(1, 20, use_graph=False)
        flat = [s.flatness() for s in systems]
        if all(f[0] > 0 and f[0] >= 0.5 * f[1] for f in flat):
            break
    else:
        pytest.fail("no flat histogram within 400 iterations")
    b.run(8, 500, use_graph=False)
    for beta, lnZ, e, c in gold:
        bp = 2 * beta
        outs = np.array([s.reweight(bp)[0] for s in systems])
        for name, est, exact in (("E/N", outs[:, 0] / N, -1.0 + e / 2), ("C/N", outs[:, 2], c),
                                 ("lnZ", outs[:, 3], bp * N + lnZ)):
            mean, err = est.mean(), est.std(ddof=1) / math.sqrt(len(est))
            assert abs(mean - exact) < 4 * err, (beta, name, mean, exact, err)
    b.close()


def _to_flat(systems, batch=None, sweeps=20, max_iter=400):
    for it in range(max_iter):
        if batch is not None:
            batch.run(1, sweeps, use_graph=False)
        else:
            for c in systems:
                c.iterate(sweeps)
                c.merge_and_update()
        flat = [s.flatness() for s in systems]
        if all(f[0] > 0 and f[0] >= 0.5 * f[1] for f in flat):
            return
    pytest.fail("no flat histogram within %d iterations" % max_iter)


def test_multimagnetic_and_energy_observables_agree():
    """Two independent routes to the canonical magnetisation of the 16x16 Ising model at
    beta = 0.4: the multimagnetic run (weights in M at fixed beta, Eq. 3, reweighted over its own
    M histogram) and MUCA in E with per-bin |M| and M^2 sums (Eq. 2).  Eight seeds each; the means
    of <|M|>/N, <M^2>/N^2 and chi/N agree within four combined standard errors."""
    beta = 0.4
    mm = [m.Muca(m.ISING2D_MUMA, 16, 2, 512, s, beta=beta) for s in range(301, 309)]
    b = m.Batch(mm)
    _to_flat(mm, b)
    b.run(8, 500, use_graph=False)
    b.close()
    a = np.array([c.reweight(beta)[0][:3] for c in mm])
    me = []
    for s in range(401, 409):
        c = m.Muca(m.ISING2D, 16, 2, 512, s)
        c.set_param("observables", 1)
        me.append(c)
    _to_flat(me)
    for _ in range(8):
        for c in me:
            c.iterate(500)
            c.merge_and_update()
    o = np.array([c.observables(beta)[0] for c in me])
    for k, name in enumerate(("<|M|>/N", "<M^2>/N^2", "chi/N")):
        ma, mo = a[:, k].mean(), o[:, k].mean()
        ea, eo = a[:, k].std(ddof=1) / math.sqrt(len(a)), o[:, k].std(ddof=1) / math.sqrt(len(o))
        assert abs(ma - mo) < 4 * math.hypot(ea, eo), (name, ma, ea, mo, eo)


def test_potts_q8_L4_density_of_states_matches_the_golden_omega():
    """8-state Potts on the 4x4 torus through the CUDA path: ln H - ln W after 12 iterations of
    4000 sweeps (1024 walkers) against the exact Omega(E) (tests/golden/potts_q8_L4_omega.txt,
    written from the transfer matrix), which spans 28 units of ln Omega over 29 reachable bins; the
    unreachable bins (1, 2, 3, 5 broken bonds) must stay unvisited.  Every bin within 0.05."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "potts_q8_L4_omega.txt")
    om = np.array([float(l.split()[1]) for l in open(path) if l.strip() and not l.startswith("#")])
    g = m.Muca(m.POTTS2D, 4, 8, 1024, 17)
    for _ in range(12):
        g.iterate(4000)
        g.merge_and_update()
    H = g.histogram()
    reach = om > 0
    assert np.all(H[~reach] == 0) and np.all(H[reach] > 0)
    lo = np.log(H[reach].astype(float)) - g.lnW_sampled()[reach]
    le = np.log(om[reach])
    d = lo + (le[0] - lo[0]) - le
    d -= d.mean()
    assert np.abs(d).max() < 0.05, np.abs(d).max()
