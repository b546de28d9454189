"""Failure detection on the GPU without a fault: the producer/consumer sweeps hand rows over
through mbarriers whose waits are bounded.  A test hook makes one producer warp leave out one
row's hand-over, so its consumer's wait runs out; the consumer then stops computing, the launch
completes, the device error flag is set and the next synchronising call returns
MUCA_ERR_TIMEOUT.  The CUDA context stays usable and the run continues from a checkpoint,
bit-exact against the oracle."""
import time

import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state

pytestmark = pytest.mark.gpu
MUCA_ERR_TIMEOUT = -4


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("system,L,q,pipeline", [(m.ISING2D, 16, 2, 2), (m.ISING2D_MUMA, 16, 2, 2),
                                                 (m.POTTS2D, 16, 5, 2), (m.ISING2D, 16, 2, 1),
                                                 (m.POTTS2D, 16, 5, 1)])
def test_bounded_wait_runs_out_and_is_reported(system, L, q, pipeline):
    beta = 0.4407 if system == m.ISING2D_MUMA else 0.0
    p = 64
    g = m.Muca(system, L, q, p, 31, beta=beta if system == m.ISING2D_MUMA else None)
    g.set_param("pipeline", pipeline)
    o = oracle.Run(system, L, q, p, 31, beta=beta)
    o.init()
    g.iterate(3)
    g.merge_and_update()
    o.iterate(3, 8)
    o.update()
    blob = g.get_state()

    g.set_param("debug_drop_row", 5)
    t0 = time.perf_counter()
    g.iterate(2)
    with pytest.raises(m.MucaError) as err:
        g.synchronize()
    elapsed = time.perf_counter() - t0
    assert err.value.code == MUCA_ERR_TIMEOUT
    assert elapsed < 120.0

    # the same context goes on from its checkpoint, bit-exact against the oracle
    g.set_state(blob)
    g.iterate(3)
    g.merge_and_update()
    o.iterate(3, 8)
    o.update()
    compare_state(g, o, "after the reported timeout and a restore")
    g.synchronize()


def test_hook_is_refused_for_the_polymer():
    g = m.Muca(m.POLYMER3D, 13, 0, 8, 1, window=(0.0, 100.0))
    with pytest.raises(m.MucaError):
        g.set_param("debug_drop_row", 1)


def test_spin_limit_bounds_the_wait():
    """The "spin_limit" parameter (and MUCA_SPIN_LIMIT at creation) sets how long a hand-over
    wait tries: a run stays healthy with a small limit, and a dropped row is reported much sooner
    than with the default bound."""
    import os

    def timed_drop(g):
        blob = g.get_state()
        g.set_param("debug_drop_row", 5)
        t0 = time.perf_counter()
        g.iterate(2)
        with pytest.raises(m.MucaError) as err:
            g.synchronize()
        assert err.value.code == MUCA_ERR_TIMEOUT
        g.set_state(blob)
        return time.perf_counter() - t0

    g = m.Muca(m.ISING2D, 16, 2, 64, 31)
    g.iterate(3)
    g.merge_and_update()
    t_default = timed_drop(g)

    s = m.Muca(m.ISING2D, 16, 2, 64, 31)
    s.set_param("spin_limit", 4096)
    o = oracle.Run(m.ISING2D, 16, 2, 64, 31)
    o.init()
    for _ in range(2):  # healthy with a small limit
        s.iterate(20)
        s.merge_and_update()
        o.iterate(20, 8)
        o.update()
    compare_state(s, o, "with spin_limit = 4096")
    s.set_param("spin_limit", 256)
    t_small = timed_drop(s)
    assert t_small < t_default / 2, (t_small, t_default)
    with pytest.raises(m.MucaError):
        s.set_param("spin_limit", -1)

    os.environ["MUCA_SPIN_LIMIT"] = "4096"
    try:
        e = m.Muca(m.ISING2D, 16, 2, 64, 31)
    finally:
        del os.environ["MUCA_SPIN_LIMIT"]
    e.iterate(3)
    e.merge_and_update()
    assert timed_drop(e) < t_default / 2
