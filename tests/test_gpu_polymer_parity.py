"""Polymer parity (Eq. 7, Eq. 2): the CUDA path against the FP64 oracle.

Trajectories.  Both sides record every attempt (the GPU through muca_poly_trace, the oracle in its
own trace).  Coordinates live on an exact grid on both sides, so walkers that make the same
decisions stay bit-identical; the GPU's pair terms are FP32, so a decision may differ only where the
oracle flags an event (a near tie of the acceptance test, an energy within the FP32 error bound of a
bin edge, a walk-in distance tie, a bond about to break).  For every walker and every call the test
finds the first attempt at which the accept decision or the bin after it differs, and requires
  - that attempt to be an event the oracle flagged (so every walker agrees bit for bit at least up to
    its first event, and no walker is left out);
  - before it: each energy change within 1e-6 * S (S = the sum of |v| + |r v'| over the move's old
    and new pair terms, plus 2^-27 for the fixed-point rounding), and the GPU's running energy within
    the oracle's bound delta of the oracle's;
  - if a walker never disagrees within a call: identical coordinates at its end and the same bin,
    unless the closing energy refresh puts the energy within its bound of a bin edge.
Weights: after each update the GPU's ln W must equal the oracle's bit for bit when the histograms
agree; in any case the oracle's ln W is then given to the GPU (muca_set_lnW), so every call of the
run is compared under identical, non-trivial weights.  Walkers that diverged stay out of later calls.
The measured |dE_gpu - dE_oracle| / S over all compared attempts is printed per case.

Density of states.  The GPU's ln H - ln W after 12 multicanonical iterations against the oracle's
from independent seeds (16 each), bin by bin within their combined standard error; and the N = 3
chain against its density of states by quadrature (both models, with and without rotations)."""
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
WINDOWS = {0: _WJ["windows"], 1: _WJ["paper_model"]["windows"]}
TAU = 1e-6
RHO = 32 * 2.0 ** -32
Q = 2.0 ** -32
NT = 8


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _pair(N, p, seed, model, moves, lanes=0, block=None, window=None, grid=(10, 1229)):
    lo, hi = window if window else (WINDOWS[model][str(N)]["e_lo"], WINDOWS[model][str(N)]["e_hi"])
    g = m.Muca(m.POLYMER3D, N, 0, p, seed, window=(lo, hi), block=block)
    if grid != (10, 1229):  # bins of width 1/k, moves in a cube of side step_q / 4096
        g.set_param("bin_width", 1.0 / grid[0])
        g.set_param("step", grid[1] / 4096.0)
    if model:
        g.set_param("model", model)
    if moves:
        g.set_param("moves", moves)
    if lanes:
        g.set_param("lanes", lanes)
    o = oracle.PolyRun(N, p, seed, lo, hi, model=model, moves=moves, bin_k=grid[0], step_q=grid[1])
    o.init()
    return g, o, lo


def compare_call(tg, to, g, o, lo, alive, stats, what, k=10):
    """Compare one call's traces walker by walker (see the module docstring); updates `alive`."""
    compare_arrays(tg, to, g.coords(), o.coords(), g.bins(), o.bins(), o.energy(), o.delta(), lo, alive, stats,
                   what, k)


def compare_arrays(tg, to, Xg, Xo, bins_g, bins_o, E_end, d_end, lo, alive, stats, what, k=10):
    """compare_call on arrays: traces (walkers, sweeps, N), end coordinates and bins of both sides,
    the oracle's refreshed energies and bounds, all for the same walkers in the same order."""
    p = tg.shape[0]
    flat = lambda a: a.reshape(p, -1)
    acc_g, acc_o = flat(tg["flags"]) & 1, flat(to["flags"]) & 1
    bg, bo = flat(tg["b"]), flat(to["bin_after"])
    dis = (acc_g != acc_o) | (bg != bo)
    first = np.where(dis.any(axis=1), np.argmax(dis, axis=1), -1)
    fo = flat(to["flags"])
    dq, dE, sc = flat(tg["dq"]) * Q, flat(to["dE"]), flat(to["scale"])
    Eg, Eo, dl = flat(tg["E"]) * Q, flat(to["E"]), flat(to["delta"])
    gbad = (flat(tg["flags"]) & 6) != 0
    for w in np.nonzero(alive)[0]:
        n = first[w] if first[w] >= 0 else dis.shape[1]
        ok = np.isfinite(dE[w, :n]) & ~gbad[w, :n]
        err = np.abs(dq[w, :n][ok] - dE[w, :n][ok])
        assert np.all(err <= TAU * sc[w, :n][ok] + RHO), "%s: walker %d, energy change beyond 1e-6 S" % (what, w)
        pos = sc[w, :n][ok] > 0
        stats["ratio"].append(err[pos] / sc[w, :n][ok][pos])
        eerr = np.abs(Eg[w, :n] - Eo[w, :n])
        assert np.all(eerr <= dl[w, :n] + 1e-9), "%s: walker %d, running energy beyond its bound" % (what, w)
        stats["energy"].append(eerr / dl[w, :n])
        stats["compared"] += int(n)
        if first[w] >= 0:
            assert fo[w, n] & 4, "%s: walker %d disagrees at attempt %d, which is not an event" % (what, w, n)
            stats["diverged"] += 1
            alive[w] = False
        else:
            np.testing.assert_array_equal(Xg[w], Xo[w], err_msg="%s: walker %d coordinates" % (what, w))
            if bins_g[w] != bins_o[w]:   # only the closing refresh may move the bin, within its bound
                t = (E_end[w] - lo) * k
                assert abs(t - round(t)) < k * d_end[w], "%s: walker %d bin after the refresh" % (what, w)
                stats["diverged"] += 1
                alive[w] = False
    stats["attempts"] += int(alive.size * dis.shape[1])


CASES = [  # N, lanes, walkers, block, model, moves, sweeps of each call (the first walks in)
    (13, 16, 64, None, 0, 0, [100, 30, 30]),
    (13, 8, 45, 160, 0, 0, [100, 30, 30]),
    (13, 32, 37, 96, 0, 0, [100, 30, 30]),
    (32, 16, 64, None, 0, 0, [120, 20, 20]),
    (32, 8, 61, None, 0, 0, [120, 20, 20]),
    (32, 32, 64, None, 0, 0, [120, 20, 20]),
    (64, 16, 64, None, 0, 0, [100, 10, 10]),
    (128, 16, 32, None, 0, 0, [100, 8, 8]),
    (128, 32, 29, 96, 0, 0, [100, 8, 8]),
    (128, 8, 33, None, 0, 0, [100, 8, 8]),
    (40, 16, 48, None, 1, 0, [100, 20, 20]),   # the paper's parameters
    (13, 16, 48, None, 0, 1, [100, 20, 20]),   # shifts and spherical rotations
    (40, 16, 48, None, 1, 1, [100, 20, 20]),
]


@pytest.mark.parametrize("N,lanes,p,block,model,moves,calls", CASES)
def test_trajectories_agree_until_the_first_event(N, lanes, p, block, model, moves, calls):
    g, o, lo = _pair(N, p, 9, model, moves, lanes, block)
    np.testing.assert_array_equal(g.coords(), o.coords())
    assert np.all(np.abs(g.energies() - o.energy()) <= o.delta())
    alive = np.ones(p, dtype=bool)
    stats = {"ratio": [], "energy": [], "compared": 0, "attempts": 0, "diverged": 0}
    same_h = True   # every histogram so far identical: the recursion's accumulated state is too
    for k, S in enumerate(calls):
        tg = g.iterate_traced(S)
        to = o.iterate_traced(S, NT)
        compare_call(tg, to, g, o, lo, alive, stats, "call %d" % k)
        g.merge_and_update()
        o.update()
        same_h = same_h and np.array_equal(g.histogram(), o.histogram())
        if same_h:
            np.testing.assert_array_equal(g.lnW().view(np.uint64), o.lnW().view(np.uint64))
        g.set_lnW(o.lnW())
    r = np.concatenate(stats["ratio"]) if stats["ratio"] else np.zeros(1)
    e = np.concatenate(stats["energy"])
    print("\nN=%d lanes=%d model=%d moves=%d: %d of %d attempts compared, %d walkers diverged at events; "
          "|dE_gpu - dE_oracle| / S: max %.3g, 99.9%% %.3g, median %.3g over %d attempts; "
          "|E_gpu - E_oracle| / delta: max %.3g"
          % (N, lanes or 16, model, moves, stats["compared"], stats["attempts"], stats["diverged"], r.max(),
             np.quantile(r, 0.999), np.median(r), r.size, e.max()))
    # most of the run is compared, not excused
    assert stats["compared"] > 0.5 * stats["attempts"]
    assert r.max() <= TAU


@pytest.mark.parametrize("N,grid,calls", [(13, (5, 614), [150, 30, 30]), (32, (20, 2048), [150, 20, 20])])
def test_trajectories_with_other_bins_and_steps(N, grid, calls):
    """Bins of width 0.2 and moves in a cube of side 0.15 (N = 13); bins of 0.05 and a cube of
    side 0.5 (N = 32): the same trajectory rule as above."""
    p = 48
    g, o, lo = _pair(N, p, 17, 0, 0, grid=grid)
    assert g.B == o.B == round((WINDOWS[0][str(N)]["e_hi"] - lo) * grid[0])
    alive = np.ones(p, dtype=bool)
    stats = {"ratio": [], "energy": [], "compared": 0, "attempts": 0, "diverged": 0}
    for k, S in enumerate(calls):
        tg = g.iterate_traced(S)
        to = o.iterate_traced(S, NT)
        compare_call(tg, to, g, o, lo, alive, stats, "call %d" % k, grid[0])
        g.merge_and_update()
        o.update()
        g.set_lnW(o.lnW())
    r = np.concatenate(stats["ratio"])
    assert stats["compared"] > 0.5 * stats["attempts"]
    assert r.max() <= TAU


def test_bin_width_and_step_arguments():
    g = m.Muca(m.POLYMER3D, 13, 0, 8, 1, window=(33.3, 87.3))
    for key, bad in (("bin_width", 0.3), ("bin_width", 0.0), ("step", 0.0), ("step", 3.0)):
        with pytest.raises(m.MucaError):
            g.set_param(key, bad)
    g.set_param("bin_width", 0.25)
    assert g.B == 216
    s = m.Muca(m.ISING2D, 8, 2, 32, 1)
    with pytest.raises(m.MucaError):
        s.set_param("bin_width", 0.5)
    g.iterate(2)
    with pytest.raises(m.MucaError):
        g.set_param("step", 0.2)   # too late


def test_set_lnW_round_trip_and_errors():
    g = m.Muca(m.POLYMER3D, 13, 0, 16, 1, window=(33.3, 87.3))
    w = np.linspace(0.0, -3.0, g.B)
    g.set_lnW(w)
    np.testing.assert_array_equal(g.lnW(), w)
    with pytest.raises(m.MucaError):
        g.set_lnW(np.zeros(g.B + 1))
    bad = w.copy()
    bad[5] = np.nan
    with pytest.raises(m.MucaError):
        g.set_lnW(bad)
    s = m.Muca(m.ISING2D, 8, 2, 32, 1)
    lw = np.arange(s.B, dtype=float) * 0.1
    s.set_lnW(lw)
    got = s.lnW()
    reach = np.isfinite(got)
    np.testing.assert_array_equal(got[reach], lw[reach])
    assert (~reach).sum() == 2   # the two unreachable Ising bins stay -inf
    with pytest.raises(m.MucaError):
        m.muca_poly_trace(s.h, 256, 10)   # spin context


def _lnomega(H, lnWs, common):
    lo = np.log(H[common].astype(float)) - lnWs[common]
    return lo - lo.mean()


@pytest.mark.parametrize("N", [13, 32])
def test_density_of_states_agrees_with_oracle_over_16_seeds(N):
    """Twelve multicanonical iterations (the first walks in) from 16 seeds on each side, seeds not
    shared: per bin, the GPU's mean ln H - ln W and the oracle's agree within their combined
    standard error (every |z| < 6 and mean z^2 < 2 over the bins all 32 runs visited >= 50 times)."""
    p, S, iters = 64, 150 if N == 13 else 100, 12
    lo, hi = WINDOWS[0][str(N)]["e_lo"], WINDOWS[0][str(N)]["e_hi"]
    runs = {"gpu": [], "oracle": []}
    for seed in range(1, 17):
        g = m.Muca(m.POLYMER3D, N, 0, p, seed, window=(lo, hi))
        o = oracle.PolyRun(N, p, 1000 + seed, lo, hi)
        o.init()
        for it in range(iters):
            g.iterate(S)
            g.merge_and_update()
            o.iterate(S, NT)
            o.update()
        runs["gpu"].append((g.histogram(), g.lnW_sampled()))
        runs["oracle"].append((o.histogram(), o.lnW_sampled()))
    common = np.all([H >= 50 for side in runs.values() for H, _ in side], axis=0)
    assert common.sum() > 100
    est = {k: np.array([_lnomega(H, lw, common) for H, lw in v]) for k, v in runs.items()}
    mg, mo = est["gpu"].mean(axis=0), est["oracle"].mean(axis=0)
    se = np.sqrt(est["gpu"].var(axis=0, ddof=1) / 16 + est["oracle"].var(axis=0, ddof=1) / 16)
    z = (mg - mo) / se
    print("\nN=%d: %d bins, max |z| %.2f, mean z^2 %.2f, max |mean difference| %.4f"
          % (N, common.sum(), np.abs(z).max(), (z * z).mean(), np.abs(mg - mo).max()))
    assert np.abs(z).max() < 6.0 and (z * z).mean() < 2.0


@pytest.mark.parametrize("model,moves", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_trimer_density_of_states_by_quadrature(model, moves):
    """N = 3 on the GPU (two FENE bonds and the LJ pair (0, 2)): ln H - ln W over the window just
    above the lowest energy against the binned density of states by quadrature, within 0.05 in
    every bin, in both parameter sets and with rotations.  1024 walkers (16 times the oracle's
    statistics for the same test), so the estimate's own noise stays well inside the bound."""
    if model == 0:
        e_lo, e_hi, sweeps, final = 10.7, 18.7, 12000, 0
        omega_args = dict(K=40.0, R=1.5, rc=2.5)
    else:
        e_lo, e_hi, sweeps, final = -0.9, 7.1, 6000, 30000
        omega_args = dict(K=40.0, R=0.3, rc=None, r0=0.7, sigma=2.0 ** (-1.0 / 6.0) * 0.7)
    g = m.Muca(m.POLYMER3D, 3, 0, 1024, 13, window=(e_lo, e_hi))
    if model:
        g.set_param("model", model)
    if moves:
        g.set_param("moves", moves)
    for _ in range(14):
        g.iterate(sweeps)
        g.merge_and_update()
    if final:
        g.iterate(final)
        g.merge_and_update()
    edges = [e_lo + 0.1 * b for b in range(g.B + 1)]
    omega = np.array(ex.fene_lj_trimer_omega(edges, **omega_args))
    H = g.histogram().astype(float)
    assert np.all(H > 0)
    lo_ = np.log(H) - g.lnW_sampled()
    le = np.log(omega)
    d = lo_ + np.median(le - lo_) - le
    print("\nmodel %d moves %d: max |d| %.4f rms %.4f" % (model, moves, np.abs(d).max(), np.sqrt((d * d).mean())))
    assert np.max(np.abs(d)) < 0.05 and np.sqrt(np.mean(d * d)) < 0.02



@pytest.mark.parametrize("N,calls", [(13, [100, 20]), (128, [80, 4])])
def test_full_size_sampled_walkers_in_the_bench_configuration(N, calls):
    """The bench's configuration (p = 4096, 256-thread blocks, 16 lanes a walker, pilot window): the
    GPU runs all walkers with tracing; the oracle runs only 24 walkers spread over the launch (the
    first and last, block and warp edges, odd positions), one at a time.  Each sampled walker agrees
    up to its first disagreement, which must be an oracle-flagged event, as in the cases above.  The
    second call runs under non-trivial weights: the oracle's update from the sampled walkers'
    histogram, given to the GPU."""
    p = 4096
    lo, hi = WINDOWS[0][str(N)]["e_lo"], WINDOWS[0][str(N)]["e_hi"]
    g = m.Muca(m.POLYMER3D, N, 0, p, 5, window=(lo, hi))
    o = oracle.PolyRun(N, p, 5, lo, hi)
    o.init()
    sample = np.array([0, 1, 15, 16, 17, 31, 32, 33, 511, 512, 1000, 1023, 1024, 2047, 2048, 2049, 2500,
                       3071, 3072, 3583, 4000, 4093, 4094, 4095])
    np.testing.assert_array_equal(g.coords()[sample], o.coords()[sample])
    alive = np.ones(sample.size, dtype=bool)
    stats = {"ratio": [], "energy": [], "compared": 0, "attempts": 0, "diverged": 0}
    for k, S in enumerate(calls):
        tg = g.iterate_traced(S, walkers=sample)
        to = np.concatenate([o.iterate_range_traced(S, int(w), int(w) + 1) for w in sample])
        o.advance(S)
        compare_arrays(tg, to, g.coords()[sample], o.coords()[sample], g.bins()[sample], o.bins()[sample],
                       o.energy()[sample], o.delta()[sample], lo, alive, stats, "call %d" % k)
        g.merge_and_update()
        o.update()
        g.set_lnW(o.lnW())
    r = np.concatenate(stats["ratio"])
    print("\nfull size N=%d: %d of %d sampled attempts compared, %d walkers diverged at events; "
          "|dE_gpu - dE_oracle| / S max %.3g" % (N, stats["compared"], stats["attempts"], stats["diverged"], r.max()))
    assert stats["compared"] > 0.5 * stats["attempts"]
    assert r.max() <= TAU


@pytest.mark.parametrize("N,p,window,calls,floor", [
    (2, 64, (0.0, 12.0), [60, 30, 30], 0.5),           # the dimer: one bond, no Lennard-Jones pair
    (3, 61, (10.7, 18.7), [60, 30, 30], 0.5),          # the trimer window just above the ground state
    # the largest window, 12288 bins: every energy of the random-walk start lies inside, so the
    # chains stay stretched (E ~ 300, bonds near breaking, where the FENE terms' FP32 error is
    # largest) and events, hence divergences, come sooner; a smaller share is compared
    (13, 40, (33.3, 33.3 + 1228.8), [100, 20], 0.1),
])
def test_trajectories_degenerate_chains_and_the_largest_window(N, p, window, calls, floor):
    """Same rule as above at the edges: every walker agrees up to its first disagreement, which
    must be a flagged event."""
    g, o, lo = _pair(N, p, 3, 0, 0, window=window)
    assert g.B == o.B and (N != 13 or g.B == 12288)
    alive = np.ones(p, dtype=bool)
    stats = {"ratio": [], "energy": [], "compared": 0, "attempts": 0, "diverged": 0}
    for k, S in enumerate(calls):
        tg = g.iterate_traced(S)
        to = o.iterate_traced(S, NT)
        compare_call(tg, to, g, o, lo, alive, stats, "call %d" % k)
        g.merge_and_update()
        o.update()
        g.set_lnW(o.lnW())
    assert stats["compared"] > floor * stats["attempts"]
    r = np.concatenate(stats["ratio"])
    assert r.max() <= TAU


def test_window_beyond_the_largest_is_refused():
    g = m.Muca(m.POLYMER3D, 13, 0, 8, 1, window=(33.3, 33.3 + 1228.8))   # 12288 bins: accepted
    assert g.B == 12288
    with pytest.raises(m.MucaError) as e:
        g.set_param("e_hi", 33.3 + 1228.9)                               # 12289 bins
    assert e.value.code == -6
