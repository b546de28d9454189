"""Pins of the oracle's per-iteration metrics (accepted moves, tunnelling events).

The oracle counts inside its sweep loop.  These tests derive the same numbers from outside it:
* with ln W = 0 every threshold is "always", so the first iteration accepts every attempt;
* a site is visited once per sweep and an accepted move always changes it (the Potts proposal
  differs from the old colour), so a sweep's accepted moves are the sites whose spin differs
  before and after it;
* tunnelling events follow from the walkers' bins at the end of each sweep by the definition
  (an arrival at the lowest reachable bin after the highest was the last end visited, or the
  reverse), restated here with its own state machine.
"""
import numpy as np
import pytest

import oracle

ISING, POTTS, MUMA = 0, 1, 2


def _tunnel_events(bin_seq, lo, hi):
    """bin_seq: (sweeps, p) bins at the end of each sweep.  Returns events per walker and the
    final 'last end' of each walker (0 none, 1 lowest, 2 highest)."""
    sweeps, p = bin_seq.shape
    last = np.zeros(p, dtype=np.int64)
    ev = np.zeros(p, dtype=np.int64)
    for s in range(sweeps):
        for w in range(p):
            b = bin_seq[s, w]
            if b == lo:
                if last[w] == 2:
                    ev[w] += 1
                last[w] = 1
            elif b == hi:
                if last[w] == 1:
                    ev[w] += 1
                last[w] = 2
    return ev, last


@pytest.mark.parametrize("system,L,q", [(ISING, 8, 2), (POTTS, 8, 5), (MUMA, 8, 2)])
def test_first_iteration_accepts_everything(system, L, q):
    """MUCA in E with ln W = 0, and MUMA at beta = 0 (its Boltzmann factor is 1): every
    threshold is "always"."""
    p, sweeps = 12, 30
    o = oracle.Run(system, L, q, p, 11, beta=0.0)
    o.init()
    o.iterate(sweeps, 2)
    o.update()
    m = o.metrics()
    assert int(m[0]) == p * L * L * sweeps
    assert int(m[4]) == sweeps
    assert int(m[2]) == int(m[0]) and int(m[3]) == int(m[1])


@pytest.mark.parametrize("system,L,q", [(ISING, 4, 2), (POTTS, 4, 3), (MUMA, 4, 2)])
def test_recount_sweep_by_sweep(system, L, q):
    """Iterations of single-sweep calls: accepted = changed sites per sweep, events from the
    per-sweep bins; several iterations so that the weights flatten and walkers tunnel."""
    p = 16
    o = oracle.Run(system, L, q, p, 3, beta=0.44)
    o.init()
    reach = np.flatnonzero(o.reachable())
    lo, hi = int(reach[0]), int(reach[-1])
    total_acc = total_ev = 0
    bins_all = []
    for it in range(12):
        sweeps = 40
        acc = 0
        for _ in range(sweeps):
            before = o.spins().copy()
            o.iterate(1, 1)
            after = o.spins()
            acc += int(np.count_nonzero(before != after))
            bins_all.append(o.bins().copy())
        o.update()
        m = o.metrics()
        ev_now, _ = _tunnel_events(np.array(bins_all), lo, hi)
        ev_it = int(ev_now.sum()) - total_ev
        assert int(m[0]) == acc, it
        assert int(m[1]) == ev_it, it
        assert int(m[4]) == sweeps
        total_acc += acc
        total_ev += ev_it
        assert int(m[2]) == total_acc and int(m[3]) == total_ev
    # L = 4 walkers cross the whole range within these iterations: the count is exercised
    assert total_ev > 0


def test_tunnel_state_machine_examples():
    """The restated definition on hand-made bin sequences (lowest 0, highest 9)."""
    seq = np.array([[5], [0], [3], [9], [9], [4], [0], [0], [9]])
    ev, last = _tunnel_events(seq, 0, 9)
    assert ev[0] == 3 and last[0] == 2
    seq = np.array([[9], [9], [5]])  # a start at an end is no event
    ev, last = _tunnel_events(seq, 0, 9)
    assert ev[0] == 0 and last[0] == 2


def test_polymer_metrics_totals():
    """Polymer: first-iteration acceptance below 1 (overlaps and FENE breaks are rejected),
    totals are the sums of the closed iterations, sweeps are counted."""
    o = oracle.PolyRun(8, 6, 5, -8.0, 40.0)
    o.init()
    tot = np.zeros(2, dtype=np.int64)
    for it in range(3):
        o.iterate(20, 2)
        o.update()
        m = o.metrics().astype(np.int64)
        assert m[4] == 20
        assert 0 < m[0] <= 6 * 8 * 20
        tot += m[:2]
        assert m[2] == tot[0] and m[3] == tot[1]
