"""The no-allocation entry point muca_iterate_noalloc, for callers that cannot call cudaMalloc
while they run an iteration (graph capture, restricted memory pools, memory-limited processes).

It must give the same histogram and the same walker states as the allocating path
(muca_iterate + muca_merge_and_update) on two calls in a row; integer histograms are compared
exactly, as everywhere in these tests.  This file is collected last on purpose."""
import numpy as np
import pytest

import paper_1312_2213_gb300 as m

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("system,L,q,p", [(m.ISING2D, 32, 2, 1000), (m.POTTS2D, 16, 10, 300),
                                          (m.ISING2D_MUMA, 16, 2, 257), (m.POTTS2D, 64, 8, 40)])
def test_noalloc_matches_allocating_path_on_two_calls(system, L, q, p):
    """Also q-Potts at L = 64, whose code form keeps only the thresholds' upper halves in shared
    memory."""
    import torch

    S = 150 if L < 64 else 4
    beta = 0.4407 if system == m.ISING2D_MUMA else None
    ref1 = m.Muca(system, L, q, p, 77, beta=beta)   # one iterate, then merge
    ref2 = m.Muca(system, L, q, p, 77, beta=beta)   # two iterates, then one merge
    nal = m.Muca(system, L, q, p, 77, beta=beta)
    dH = torch.full((nal.B,), -1, dtype=torch.int64, device="cuda")  # stale contents must be overwritten

    ref1.iterate(S)
    ref1.merge_and_update()
    m.muca_iterate_noalloc(nal.h, S, dH.data_ptr())
    nal.synchronize()
    h1 = dH.cpu().numpy().view(np.uint64).copy()
    np.testing.assert_array_equal(h1, ref1.histogram())
    np.testing.assert_array_equal(nal.spins(), ref1.spins())
    np.testing.assert_array_equal(nal.bins(), ref1.bins())

    ref2.iterate(S)
    ref2.iterate(S)
    ref2.merge_and_update()
    m.muca_iterate_noalloc(nal.h, S, dH.data_ptr())
    nal.synchronize()
    h2 = dH.cpu().numpy().view(np.uint64).copy()
    np.testing.assert_array_equal(h1 + h2, ref2.histogram())
    np.testing.assert_array_equal(nal.spins(), ref2.spins())
    np.testing.assert_array_equal(nal.bins(), ref2.bins())
    assert nal.sweep_counter() == 2 * S
    assert int(h2.sum()) == p * S * L * L
    # the no-alloc sweeps count toward the next closed iteration's metrics, like any sweeps
    nal.merge_and_update()
    mn, mr = nal.metrics(), ref2.metrics()
    assert mn["sweeps"] == mr["sweeps"] == 2 * S
    assert mn["accepted"] == mr["accepted"] > 0
    assert mn["tunnelling_events"] == mr["tunnelling_events"]


def test_noalloc_records_no_observables():
    """Observable sums are recorded by muca_iterate only: an iteration made of no-alloc sweeps
    closes with empty sums."""
    import torch

    g = m.Muca(m.ISING2D, 16, 2, 64, 9)
    g.set_param("observables", 1)
    g.iterate(20)
    g.merge_and_update()
    _, sums = g.observables(0.4)
    assert int(sums[:, 0].sum()) == 64 * 20
    dH = torch.zeros(g.B, dtype=torch.int64, device="cuda")
    m.muca_iterate_noalloc(g.h, 20, dH.data_ptr())
    g.merge_and_update()
    _, sums = g.observables(0.4)
    assert int(sums.sum()) == 0
    assert int(dH.sum()) == 64 * 20 * 256


def test_noalloc_rejects_sizes_beyond_the_static_array():
    import torch

    big = m.Muca(m.ISING2D_MUMA, 64, 2, 8192, 1, beta=0.4407)  # 128 blocks x 4097 bins > 2^19 slots
    dH = torch.zeros(big.B, dtype=torch.int64, device="cuda")
    with pytest.raises(m.MucaError) as e:
        m.muca_iterate_noalloc(big.h, 1, dH.data_ptr())
    assert e.value.code == -6
    assert "static maximum" in str(e.value)
