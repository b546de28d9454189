"""GPU polymer path (8, 16 or 32 lanes per walker, FP32 pair terms, exact fixed-point sums) against the
FP64 oracle: initial chains, the all-accepting first iteration, the FENE dimer's closed form,
reweighting, checkpoints and the paper's parameter set.  Trajectory parity attempt by attempt and
the density of states against the oracle are in test_gpu_polymer_parity.py.  Coordinates live on a
2^-44 grid on both sides, so trajectories that make the same accept/reject decisions are
bit-identical.  Tolerance for energies: 1e-6 of the sum of |pair energies| (FP32 pair terms)."""
import json
import os

import numpy as np
import pytest

import oracle
import oracle.exact as ex
import paper_1312_2213_gb300 as m

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
_WJ = json.load(open(os.path.join(ROOT, "paper_1312_2213_gb300", "polymer_windows.json")))
WINDOWS = _WJ["windows"]
PAPER_WINDOWS = _WJ["paper_model"]["windows"]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def energy_scale(X, model=0):
    """Sum over pairs of |pair energy| (the scale of the FP32 rounding of an energy)."""
    N = X.shape[0]
    s = 0.0
    for i in range(N):
        for j in range(i + 1, N):
            s += abs(oracle.poly_pair(float(np.linalg.norm(X[i] - X[j])), j - i, model))
    return s


@pytest.mark.parametrize("N", [2, 13, 32, 64, 128])
def test_init_chains_bit_exact(N):
    p = 40
    lo, hi = (0.0, 12.0) if N == 2 else (WINDOWS[str(N)]["e_lo"], WINDOWS[str(N)]["e_hi"])
    g = m.Muca(m.POLYMER3D, N, 0, p, 21, window=(lo, hi))
    o = oracle.PolyRun(N, p, 21, lo, hi)
    o.init()
    np.testing.assert_array_equal(g.coords(), o.coords())
    ge, oe = g.energies(), o.energy()
    for w in range(0, p, 7):
        assert abs(ge[w] - oe[w]) <= 1e-6 * energy_scale(o.coords()[w]) + 1e-9


def test_first_iteration_trajectories_identical():
    """ln W = 0 and a window containing every reachable energy: every move that keeps the bonds
    intact is accepted on both sides, so all chains must stay bit-identical (the moves are exact
    grid arithmetic) and the energies must agree within the FP32 tolerance.  With every move
    accepted the chains wander into steep overlapping Lennard-Jones contacts, so the histograms
    are compared in the realistic window below, not here."""
    N, p, S = 13, 48, 60
    lo, hi = 0.0, 1000.0
    g = m.Muca(m.POLYMER3D, N, 0, p, 5, window=(lo, hi))
    o = oracle.PolyRun(N, p, 5, lo, hi)
    o.init()
    g.iterate(S)
    g.merge_and_update()
    o.iterate(S, 8)
    o.update()
    np.testing.assert_array_equal(g.coords(), o.coords())
    gX = o.coords()
    ge, oe = g.energies(), o.energy()
    for w in range(p):
        assert abs(ge[w] - oe[w]) <= 1e-6 * energy_scale(gX[w]) + 1e-9
    assert int(g.histogram().sum()) == int(o.histogram().sum()) == p * S * N


def test_fene_dimer_matches_closed_form():
    """N = 2 on the GPU: multicanonical estimate of the binned density of states against the
    closed form (4 pi/3)(r(E_b)^3 - r(E_a)^3)."""
    lo, hi = 0.0, 12.0
    g = m.Muca(m.POLYMER3D, 2, 0, 4096, 11, window=(lo, hi))
    for _ in range(10):
        g.iterate(200)
        g.merge_and_update()
    H = g.histogram().astype(float)
    seen = H > 0
    assert seen.mean() > 0.98
    edges = [lo + 0.1 * b for b in range(g.B + 1)]
    om = np.array(ex.fene_dimer_omega(edges, 40.0, 1.5))
    lo_ = np.log(H[seen]) - g.lnW_sampled()[seen]
    le = np.log(om[seen])
    assert np.max(np.abs(lo_ + np.median(le - lo_) - le)) < 0.1


def test_polymer_reweight_matches_oracle():
    """Eq. (2) on the polymer: identical results where the histograms agree, close otherwise."""
    N, p, S = 13, 64, 40
    lo, hi = WINDOWS[str(N)]["e_lo"], WINDOWS[str(N)]["e_hi"]
    g = m.Muca(m.POLYMER3D, N, 0, p, 7, window=(lo, hi))
    o = oracle.PolyRun(N, p, 7, lo, hi)
    o.init()
    g.iterate(S)
    g.merge_and_update()
    o.iterate(S, 8)
    o.update()
    same_h = np.array_equal(g.histogram(), o.histogram())
    for beta in (0.2, 1.0):
        go, _ = g.reweight(beta)
        oo, _ = o.reweight(beta)
        np.testing.assert_allclose(go, oo, rtol=1e-10 if same_h else 1e-2, atol=1e-10 if same_h else 1e-2)


def test_polymer_checkpoint_resume_bit_exact():
    lo, hi = WINDOWS["32"]["e_lo"], WINDOWS["32"]["e_hi"]
    a = m.Muca(m.POLYMER3D, 32, 0, 100, 3, window=(lo, hi))
    for _ in range(4):
        a.iterate(20)
        a.merge_and_update()
    b = m.Muca(m.POLYMER3D, 32, 0, 100, 3, window=(lo, hi))
    for _ in range(2):
        b.iterate(20)
        b.merge_and_update()
    st = b.get_state()
    c = m.Muca(m.POLYMER3D, 32, 0, 100, 3)     # default window: restored from the state
    c.set_state(st)
    c.B = m.muca_num_bins(c.h)
    for _ in range(2):
        c.iterate(20)
        c.merge_and_update()
    np.testing.assert_array_equal(a.coords(), c.coords())
    np.testing.assert_array_equal(a.histogram(), c.histogram())
    np.testing.assert_array_equal(a.lnW(), c.lnW())


def test_polymer_argument_errors():
    with pytest.raises(m.MucaError):
        m.Muca(m.POLYMER3D, 129, 0, 10, 1)
    g = m.Muca(m.POLYMER3D, 13, 0, 10, 1)
    with pytest.raises(m.MucaError) as e:
        g.set_param("e_hi", 1e6)   # too many bins
    assert e.value.code == -6
    with pytest.raises(m.MucaError):
        g.spins()
    with pytest.raises(m.MucaError):
        g.set_param("fene_R", -1.0)


@pytest.mark.parametrize("N", [40, 80])
def test_paper_model_init_bit_exact(N):
    """Model 1 (the paper's Eq. 7 parameters): initial chains with bonds r0 = 0.7 are bit-identical
    to the oracle's, energies within the FP32 tolerance."""
    p = 24
    lo, hi = PAPER_WINDOWS[str(N)]["e_lo"], PAPER_WINDOWS[str(N)]["e_hi"]
    g = m.Muca(m.POLYMER3D, N, 0, p, 23, window=(lo, hi))
    g.set_param("model", 1)
    o = oracle.PolyRun(N, p, 23, lo, hi, model=1)
    o.init()
    np.testing.assert_array_equal(g.coords(), o.coords())
    ge, oe = g.energies(), o.energy()
    for w in range(0, p, 5):
        assert abs(ge[w] - oe[w]) <= 1e-6 * energy_scale(o.coords()[w], 1) + 1e-9


def test_paper_model_state_round_trip():
    """The model travels with the checkpoint."""
    g = m.Muca(m.POLYMER3D, 40, 0, 8, 3, window=(PAPER_WINDOWS["40"]["e_lo"], PAPER_WINDOWS["40"]["e_hi"]))
    g.set_param("model", 1)
    g.iterate(3)
    g.merge_and_update()
    st = g.get_state()
    h = m.Muca(m.POLYMER3D, 40, 0, 8, 3)
    h.set_state(st)
    np.testing.assert_array_equal(g.coords(), h.coords())
    g.iterate(2)
    h.iterate(2)
    np.testing.assert_array_equal(g.coords(), h.coords())
