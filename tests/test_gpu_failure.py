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
