"""Pins of the polymer oracle's event rule, the part of the oracle that says where an implementation
with lower-precision pair terms may decide differently (trajectory parity of the polymer, Eq. 7).

The rule: a run whose pair terms are within tau * sigma(r) of the exact ones (sigma = |v| + |r v'|)
makes the oracle's decisions at every attempt the oracle does not flag as an event.  Checked here
against a planted error in the oracle itself: a second oracle run whose every pair term is moved by
up to tau * sigma must diverge from the clean run only at attempts the clean run flagged, while a
planted error 300 times larger produces divergences the rule did not flag (so the check can fail).
The error scale sigma is checked against its definition by numerical differentiation."""
import json
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WINDOWS = json.load(open(os.path.join(ROOT, "paper_1312_2213_gb300", "polymer_windows.json")))["windows"]
TAU = 1e-6


@pytest.mark.parametrize("model", [0, 1])
def test_error_scale_is_value_plus_r_times_derivative(orc, model):
    """FENE: sigma = |v| + |r v'| (v' by central differences).  LJ: the same taken over its two
    parts, 4 (s^12 + s^6) + 4 (12 s^12 + 6 s^6) with s = sigma_LJ / r (plus |shift| for the shifted
    potential), which is never below |v| + |r v'|."""
    rng = np.random.default_rng(3)
    sig = 0.7 * 2 ** (-1 / 6) if model == 1 else 1.0
    shift = 0.0 if model == 1 else 4 * abs(2.5 ** -12 - 2.5 ** -6)
    r_lj = rng.uniform(0.85, 2.45, 40) * sig
    r_fene = rng.uniform(0.41, 0.99, 40) if model == 1 else rng.uniform(0.2, 1.49, 40)
    for sep, rs in ((2, r_lj), (1, r_fene)):
        for r in rs:
            h = 1e-6 * r
            dv = (orc.poly_pair(r + h, sep, model) - orc.poly_pair(r - h, sep, model)) / (2 * h)
            first_order = abs(orc.poly_pair(r, sep, model)) + abs(r * dv)
            got = orc.poly_pair_scale(r, sep, model)
            if sep == 1:
                assert got == pytest.approx(first_order, rel=1e-5), (sep, r)
            else:
                s6 = (sig / r) ** 6
                assert got == pytest.approx(4 * (13 * s6 * s6 + 7 * s6) + shift, rel=1e-12), (sep, r)
                assert got >= first_order * (1 - 1e-6)
    assert orc.poly_pair_scale(2.6, 2, 0) == 0.0                   # beyond the cutoff
    assert orc.poly_pair_scale(1.5, 1, 0) == float("inf")          # broken bond


def _run(orc, N, p, seed, calls, perturb=0.0, model=0, windows=WINDOWS):
    """Run a clean oracle A and, if perturb > 0, a perturbed oracle B on the same seeds, call by call,
    giving B A's weights after every update.  Returns per call the two traces (B's None if clean)."""
    lo, hi = windows[str(N)]["e_lo"], windows[str(N)]["e_hi"]
    A = orc.PolyRun(N, p, seed, lo, hi, model=model)
    B = orc.PolyRun(N, p, seed, lo, hi, model=model)
    B.set_perturbation(perturb)
    A.init()
    B.init()
    out = []
    for S in calls:
        ta = A.iterate_traced(S, 8)
        tb = B.iterate_traced(S, 8)
        out.append((ta, tb, A.coords(), B.coords(), A.bins(), B.bins(), A.energy(), A.delta()))
        A.update()
        B.update()
        B.set_lnW(A.lnW())
    return out


def first_disagreement(ta, tb):
    """Per walker, the first attempt (flattened sweep * N + bead) where the accept decision or the bin
    after it differs, or -1."""
    p = ta.shape[0]
    da = (ta["flags"] & 1).reshape(p, -1) != (tb["flags"] & 1).reshape(p, -1)
    db = ta["bin_after"].reshape(p, -1) != tb["bin_after"].reshape(p, -1)
    d = da | db
    k = np.argmax(d, axis=1)
    return np.where(d.any(axis=1), k, -1)


@pytest.mark.parametrize("N", [13, 32])
def test_planted_error_within_the_bound_diverges_only_at_flagged_events(orc, N):
    calls = [80, 20, 20]
    res = _run(orc, N, 16, 7, calls, perturb=TAU)
    alive = np.ones(16, dtype=bool)
    checked = flagged_div = 0
    for ta, tb, Xa, Xb, ba, bb, Ea, da in res:
        k = first_disagreement(ta, tb)
        fa = ta["flags"].reshape(16, -1)
        dEa, dEb, sc = (x.reshape(16, -1) for x in (ta["dE"], tb["dE"], ta["scale"]))
        for w in np.nonzero(alive)[0]:
            n = k[w] if k[w] >= 0 else fa.shape[1]
            ok = np.isfinite(dEa[w, :n])
            # before the first disagreement the planted error of each energy change is within the bound
            assert np.all(np.abs(dEb[w, :n][ok] - dEa[w, :n][ok]) <= TAU * sc[w, :n][ok] + 1e-12)
            checked += n
            if k[w] >= 0:
                assert fa[w, k[w]] & 4, "walker %d diverged at attempt %d, which is not an event" % (w, k[w])
                flagged_div += 1
                alive[w] = False
            else:
                np.testing.assert_array_equal(Xa[w], Xb[w])
                if ba[w] != bb[w]:   # only the closing refresh may move a bin, within its bound
                    t = (Ea[w] - WINDOWS[str(N)]["e_lo"]) * 10.0
                    assert abs(t - round(t)) < 10.0 * da[w]
    assert checked > 16 * N * sum(calls) // 3
    print("N=%d: %d attempts compared, %d walkers diverged (all at flagged events)" % (N, checked, flagged_div))


def test_planted_error_beyond_the_bound_is_caught(orc):
    """300 times the tolerance: some walker diverges at an attempt that is not an event."""
    res = _run(orc, 13, 16, 7, [80, 20, 20], perturb=300 * TAU)
    unflagged = 0
    alive = np.ones(16, dtype=bool)
    for ta, tb, *_ in res:
        k = first_disagreement(ta, tb)
        fa = ta["flags"].reshape(16, -1)
        for w in np.nonzero(alive & (k >= 0))[0]:
            unflagged += int(not fa[w, k[w]] & 4)
            alive[w] = False
    assert unflagged > 0


def test_trace_agrees_with_the_run(orc):
    """The trace is the run: accepted energy changes sum to the energy change of each walker (up to
    the refresh at the end of the call), the bins after the decisions fill the histogram, and the last
    record's bin is the walker's bin unless the refresh moved it."""
    N, p, S = 13, 8, 60
    lo, hi = WINDOWS[str(N)]["e_lo"], WINDOWS[str(N)]["e_hi"]
    P = orc.PolyRun(N, p, 2, lo, hi)
    P.init()
    E0 = P.energy().copy()
    t = P.iterate_traced(S, 4)
    E1 = P.energy()
    acc = (t["flags"] & 1) == 1
    dE = np.where(acc, t["dE"], 0.0).reshape(p, -1).sum(axis=1)
    np.testing.assert_allclose(E0 + dE, E1, atol=1e-8)
    P.update()
    H = P.histogram()
    b = t["bin_after"].ravel()
    inside = (b >= 0) & (b < P.B)
    np.testing.assert_array_equal(np.bincount(b[inside], minlength=P.B).astype(np.uint64), H)
    assert np.all(t["bin_new"][acc] == t["bin_after"][acc])
    np.testing.assert_array_equal(t["bin_after"][:, -1, -1], P.bins())
    # each walker's first event is the first flagged attempt
    fe = P.first_events()
    fl = (t["flags"] & 4).reshape(p, -1) != 0
    for w in range(p):
        want = int(np.argmax(fl[w])) if fl[w].any() else -1
        assert fe[w] == want or (want == -1 and fe[w] == S * N)
