"""The flush of the sweeps' shared-memory histogram counters between chunks of sweeps.

A thread block counts its walkers' bins in uint32 shared-memory counters and adds them to its
uint64 slot every ``flush_every`` sweeps, so no counter can overflow.  The automatic chunk
(floor((2^32 - 1) / (block * N)) sweeps, 65535 at L = 32) is longer than any test run, so these
tests cap it with the "flush_every" parameter: a 10-sweep iterate with flush_every = 3 crosses
three flushes inside the launch before the final one, in every sweep form.  Histograms,
lattices, bins, thresholds and ln W must stay bit-identical to the oracle, which has no
chunks at all (the paper's merge is a plain sum of the walkers' histograms)."""
import numpy as np
import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [(m.ISING2D, 16, 2, 0.0), (m.ISING2D_MUMA, 16, 2, 0.4407), (m.POTTS2D, 16, 8, 0.0)]


@pytest.mark.parametrize("pipeline", [2, 1, 0])
@pytest.mark.parametrize("record", [0, 1])
@pytest.mark.parametrize("system,L,q,beta", CASES)
def test_flush_between_chunks_bit_exact(system, L, q, beta, pipeline, record):
    p, S = 100, 10
    g = m.Muca(system, L, q, p, 13, beta=beta if system == m.ISING2D_MUMA else None, record=record)
    g.set_param("pipeline", pipeline)
    g.set_param("flush_every", 3)
    o = oracle.Run(system, L, q, p, 13, beta=beta, record=record)
    o.init()
    for it in range(3):
        g.iterate(S)
        g.merge_and_update()
        o.iterate(S, 8)
        o.update()
        compare_state(g, o, "after iteration %d (pipeline %d)" % (it, pipeline))


@pytest.mark.parametrize("cap", [1, 2, 7])
def test_flush_cap_does_not_change_results(cap):
    """The chunk length is invisible: cap 1, 2, 7 and the automatic chunk give identical
    histograms on the default (code) form with 64-walker blocks."""
    runs = []
    for c in (0, cap):
        g = m.Muca(m.ISING2D, 32, 2, 130, 5)
        g.set_param("flush_every", c)
        g.iterate(9)
        g.merge_and_update()
        runs.append((g.histogram(), g.spins(), g.bins()))
    for a, b in zip(*runs):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("pipeline", [2, 0])
def test_flush_in_potts_L64_forms(pipeline):
    """q-Potts at L = 64: the code form with the split table (upper halves and 16-bit counters in
    shared memory) and the one-warp form with the table in global memory."""
    p, S = 40, 5
    g = m.Muca(m.POTTS2D, 64, 10, p, 3)
    g.set_param("pipeline", pipeline)
    g.set_param("flush_every", 2)
    o = oracle.Run(m.POTTS2D, 64, 10, p, 3)
    o.init()
    for it in range(2):
        g.iterate(S)
        g.merge_and_update()
        o.iterate(S, 8)
        o.update()
        compare_state(g, o, "after iteration %d" % it)


@pytest.mark.parametrize("block,record", [(64, 0), (32, 0), (64, 1)])
def test_split_counters_with_every_walker_in_one_bin(block, record):
    """q-Potts at L = 64 in the code form counts visits in 16-bit counters beside the thresholds'
    upper halves, which the consumer warps empty every F rows (F = 15 with two consumer warps a
    block, 31 with one).  Fixed weights ln W = -30 |b - b0| around the walkers' median initial bin
    b0 send every walker to b0 within the first sweep and keep it there: a move away from b0 has
    threshold 0, so only moves that keep the energy are accepted.  The counter of b0 then takes
    64 x 4096 = 2.6e5 visits a sweep, four times its range, and up to 61440 (63488) between two
    scans.  Histogram, lattices, bins and the next ln W stay bit-identical to the oracle at the
    same weights."""
    p, S, q = 64, 6, 10
    g = m.Muca(m.POTTS2D, 64, q, p, 21, record=record, block=block)
    o = oracle.Run(m.POTTS2D, 64, q, p, 21, record=record)
    o.init()
    b0 = int(np.median(o.bins()))
    lnW = -30.0 * np.abs(np.arange(g.B) - b0)
    g.set_lnW(lnW)
    o.set_lnW(lnW)
    for it in range(2):
        g.iterate(S)
        g.merge_and_update()
        o.iterate(S, 8)
        o.update()
        compare_state(g, o, "after iteration %d" % it)
        g.set_lnW(lnW)
        o.set_lnW(lnW)
    H = g.histogram()
    assert int(H.sum()) == p * S * (64 * 64 if record == 0 else 1)
    assert (g.bins() == b0).mean() > 0.9
    assert H[b0] > 0.9 * H.sum()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_flush_in_batches(form, use_graph):
    """Both batch forms (the persistent tile launch and the systems' own kernels side by side),
    plain and captured in a graph."""
    spec = [(m.ISING2D, 16, 2, 70), (m.POTTS2D, 8, 10, 50), (m.ISING2D_MUMA, 12, 2, 40)]
    gs, os_ = [], []
    for k, (system, L, q, p) in enumerate(spec):
        beta = 0.4407 if system == m.ISING2D_MUMA else 0.0
        g = m.Muca(system, L, q, p, 40 + k, beta=beta if system == m.ISING2D_MUMA else None)
        g.set_param("flush_every", 2)
        gs.append(g)
        o = oracle.Run(system, L, q, p, 40 + k, beta=beta)
        o.init()
        os_.append(o)
    b = m.Batch(gs, form=form)
    b.run(3, 5, use_graph=use_graph)
    for g in gs:
        g.synchronize()
    for g, o in zip(gs, os_):
        for _ in range(3):
            o.iterate(5, 8)
            o.update()
        compare_state(g, o, "after a batch of 3 iterations (form %d)" % form)
    b.close()


def test_flush_every_argument_checks():
    for g in (m.Muca(m.ISING2D, 8, 2, 32, 1), m.Muca(m.POLYMER3D, 13, 0, 8, 1)):
        for bad in (-1, 0.5):
            with pytest.raises(m.MucaError):
                g.set_param("flush_every", bad)
        g.set_param("flush_every", 2)


@pytest.mark.parametrize("record", [0, 1])
def test_polymer_counters_flushed_between_chunks(record):
    """The polymer sweep counts visits in a block's 32-bit shared-memory counters and adds them to
    the 64-bit histogram after every chunk; capping the chunk at 1 or 3 sweeps (7-sweep iterates
    cross several flushes in one launch) changes nothing: histogram, coordinates, energies and
    bins are identical to the run with the automatic chunk, and the histogram holds every visit."""
    runs = []
    for cap in (0, 1, 3):
        g = m.Muca(m.POLYMER3D, 13, 0, 100, 9, window=(33.3, 87.3), record=record)
        g.set_param("flush_every", cap)
        for _ in range(3):
            g.iterate(7)
            g.merge_and_update()
        H = g.histogram()
        runs.append((H, g.coords(), g.energies(), g.bins()))
    for other in runs[1:]:
        for a, b in zip(runs[0], other):
            np.testing.assert_array_equal(a, b)
    assert int(runs[0][0].sum()) > 0
