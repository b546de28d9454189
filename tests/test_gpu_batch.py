"""Batched mode: several systems in one persistent sweep launch per iteration (and the whole
run as one CUDA graph) give bit-identical results to running each context on its own, which in
turn the oracle pins; one system is also compared with the oracle directly."""
import numpy as np
import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state

pytestmark = pytest.mark.gpu

MIX = [(m.ISING2D, 16, 2, 100, 11, None), (m.POTTS2D, 16, 10, 70, 12, None), (m.ISING2D_MUMA, 8, 2, 50, 13, 0.4407),
       (m.ISING2D, 32, 2, 40, 14, None), (m.POTTS2D, 24, 10, 33, 15, None), (m.ISING2D, 64, 2, 20, 16, None)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _make():
    return [m.Muca(s, L, q, p, seed, beta=beta) for s, L, q, p, seed, beta in MIX]


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_equals_individual_runs(use_graph, form):
    n_iter, sweeps = 3, 15
    ref = _make()
    for _ in range(n_iter):
        for c in ref:
            c.iterate(sweeps)
            c.merge_and_update()
    sys_ = _make()
    b = m.Batch(sys_, form=form)
    b.run(n_iter, sweeps, use_graph=use_graph)
    b.run(2, sweeps, use_graph=use_graph)  # second run: graph re-captured for a new n_iter
    for _ in range(2):
        for c in ref:
            c.iterate(sweeps)
            c.merge_and_update()
    for r, s in zip(ref, sys_):
        np.testing.assert_array_equal(r.histogram(), s.histogram())
        np.testing.assert_array_equal(r.lnW().view(np.uint64), s.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.spins(), s.spins())
        np.testing.assert_array_equal(r.thresholds(), s.thresholds())
        assert r.sweep_counter() == s.sweep_counter() == 5 * sweeps
    b.close()


@pytest.mark.parametrize("form", [0, 1])
@pytest.mark.parametrize("use_graph", [False, True])
def test_batch_with_per_system_sweeps(use_graph, form):
    """Each system iterates at its own length (as with each system's M_opt, Eq. 4): the batch
    equals every context run alone with its own sweep count, iteration by iteration.  New counts
    re-capture the graph and reorder the launches; None restores the run's argument."""
    ref, sys_ = _make(), _make()
    b = m.Batch(sys_, form=form)

    def alone(counts, n_iter):
        for _ in range(n_iter):
            for c, sw in zip(ref, counts):
                c.iterate(sw)
                c.merge_and_update()

    total = np.zeros(len(MIX), dtype=np.int64)
    for counts, n_iter, arg in (([3, 17, 8, 25, 11, 40], 2, 5), ([7, 2, 13, 5, 9, 4], 2, 5), (None, 1, 6)):
        b.set_sweeps(counts)
        b.run(n_iter, arg, use_graph=use_graph)
        eff = counts if counts is not None else [arg] * len(MIX)
        alone(eff, n_iter)
        total += n_iter * np.asarray(eff)
    for r, s, t in zip(ref, sys_, total):
        np.testing.assert_array_equal(r.histogram(), s.histogram())
        np.testing.assert_array_equal(r.lnW().view(np.uint64), s.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.spins(), s.spins())
        assert r.sweep_counter() == s.sweep_counter() == t
    for bad in ([3] * (len(MIX) - 1), [3, 0, 3, 3, 3, 3]):
        with pytest.raises(m.MucaError):
            b.set_sweeps(bad)
    b.close()


@pytest.mark.parametrize("form", [0, 1])
def test_batch_graph_replay_matches_oracle(form):
    sys_ = _make()
    b = m.Batch(sys_, form=form)
    for _ in range(2):
        b.run(2, 10, use_graph=True)   # same graph replayed twice
    s, L, q, p, seed, beta = MIX[1]
    o = oracle.Run(s, L, q, p, seed, beta=beta or 0.0)
    o.init()
    for _ in range(4):
        o.iterate(10, 8)
        o.update()
    compare_state(sys_[1], o, "batched Potts after 4 graph iterations")


def test_batch_rejects_unmerged_and_duplicates():
    sys_ = _make()[:2]
    with pytest.raises(m.MucaError):
        m.Batch([sys_[0], sys_[0]])
    b = m.Batch(sys_)
    sys_[0].iterate(3)
    with pytest.raises(m.MucaError) as e:
        b.run(1, 5)
    assert e.value.code == -5
    sys_[0].merge_and_update()
    b.run(1, 5)


def test_batch_form_switch_keeps_results():
    """Alternating the two forms (the captured graph of one is dropped for the other) gives the
    same state as individual runs; bad form values are refused."""
    ref = _make()
    for _ in range(4):
        for c in ref:
            c.iterate(12)
            c.merge_and_update()
    sys_ = _make()
    b = m.Batch(sys_)
    b.run(1, 12, use_graph=True)
    b.set_form(1)
    b.run(1, 12, use_graph=True)
    b.set_form(0)
    b.run(1, 12, use_graph=False)
    b.set_form(1)
    b.run(1, 12, use_graph=False)
    with pytest.raises(m.MucaError):
        b.set_form(2)
    for r, c in zip(ref, sys_):
        np.testing.assert_array_equal(r.lnW().view(np.uint64), c.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.spins(), c.spins())
        assert r.metrics() == c.metrics()
    b.close()


def test_side_by_side_batch_with_mixed_forms_and_blocks():
    """Form 1 runs every system in its own configured form and block: one system per sweep form
    and several block sizes give the same results as the systems run on their own."""
    cfg = [(m.ISING2D, 16, 2, 100, 21, None, 0, 64), (m.ISING2D, 16, 2, 100, 22, None, 1, 128),
           (m.ISING2D, 16, 2, 100, 23, None, 2, 32), (m.POTTS2D, 16, 6, 90, 24, None, 2, 64),
           (m.ISING2D_MUMA, 8, 2, 70, 25, 0.4407, 1, 64)]

    def make():
        out = []
        for s, L, q, p, seed, beta, pipe, blk in cfg:
            c = m.Muca(s, L, q, p, seed, beta=beta, block=blk)
            c.set_param("pipeline", pipe)
            out.append(c)
        return out

    ref = make()
    for _ in range(3):
        for c in ref:
            c.iterate(25)
            c.merge_and_update()
    sys_ = make()
    b = m.Batch(sys_, form=1)
    b.run(3, 25, use_graph=True)
    for r, c in zip(ref, sys_):
        np.testing.assert_array_equal(r.lnW().view(np.uint64), c.lnW().view(np.uint64))
        np.testing.assert_array_equal(r.histogram(), c.histogram())
        np.testing.assert_array_equal(r.spins(), c.spins())
        assert r.metrics() == c.metrics()
    b.close()


def test_full_size_mix_bit_exact_against_the_oracle():
    """The batched mix at its benchmark size (Ising L = 16..64 and q = 10 Potts L = 16..48,
    2048 walkers each, side by side in one graph): three short iterations, every system bit-exact
    against its own oracle run."""
    mix = [(m.ISING2D, L, 2, 2048, 500 + i) for i, L in enumerate((16, 24, 32, 48, 64))] + \
          [(m.POTTS2D, L, 10, 2048, 600 + i) for i, L in enumerate((16, 24, 32, 48))]
    sys_ = [m.Muca(s, L, q, p, seed) for s, L, q, p, seed in mix]
    b = m.Batch(sys_)
    b.run(3, 4, use_graph=True)
    for (s, L, q, p, seed), c in zip(mix, sys_):
        o = oracle.Run(s, L, q, p, seed)
        o.init()
        for _ in range(3):
            o.iterate(4, 16)
            o.update()
        compare_state(c, o, "mix system %d L=%d" % (s, L))
    b.close()


def test_batch_runs_after_restoring_a_merged_checkpoint():
    """A checkpoint taken after a merge carries no unmerged counts, so a batch may run right after
    it is restored; one taken between an iterate and its merge still makes the batch refuse."""
    a = m.Muca(m.ISING2D, 16, 2, 64, 3)
    a.iterate(5)
    a.merge_and_update()
    merged = a.get_state()
    a.iterate(5)
    unmerged = a.get_state()
    c = m.Muca(m.ISING2D, 16, 2, 64, 3)
    c.set_state(merged)
    b = m.Batch([c])
    b.run(1, 5, use_graph=False)
    c.set_state(unmerged)
    with pytest.raises(m.MucaError) as e:
        b.run(1, 5, use_graph=False)
    assert e.value.code == -5
    b.close()


POLY_MIX = [(13, 64, (33.3, 87.3), 21), (32, 40, (53.0, 176.7), 22), (64, 33, (106.6, 405.7), 23)]


def _make_poly_mix():
    out = [m.Muca(m.POLYMER3D, N, 0, p, seed, window=win) for N, p, win, seed in POLY_MIX]
    out.append(m.Muca(m.ISING2D, 16, 2, 64, 24))
    return out


@pytest.mark.parametrize("use_graph", [False, True])
def test_polymer_lengths_in_one_batch(use_graph):
    """Polymers of several lengths (and a lattice system) side by side in one batch, with their
    own sweep counts: every context ends bit-identical to running alone (coordinates, energies
    refreshed from scratch, histogram, ln W), and the tile form is refused."""
    sweeps = [6, 3, 2, 20]
    ref, sys_ = _make_poly_mix(), _make_poly_mix()
    for _ in range(3):
        for c, sw in zip(ref, sweeps):
            c.iterate(sw)
            c.merge_and_update()
    b = m.Batch(sys_)
    with pytest.raises(m.MucaError):
        b.set_form(0)
    b.set_sweeps(sweeps)
    b.run(3, 1, use_graph=use_graph)
    for c in sys_:
        c.synchronize()
    for r, s in zip(ref, sys_):
        np.testing.assert_array_equal(r.histogram(), s.histogram())
        np.testing.assert_array_equal(r.lnW().view(np.uint64), s.lnW().view(np.uint64))
        assert r.sweep_counter() == s.sweep_counter()
        if r.system == m.POLYMER3D:
            np.testing.assert_array_equal(r.coords(), s.coords())
            np.testing.assert_array_equal(r.energies(), s.energies())
            np.testing.assert_array_equal(r.bins(), s.bins())
        else:
            np.testing.assert_array_equal(r.spins(), s.spins())
    b.close()
