"""GPU parity of the per-iteration metrics (accepted moves, tunnelling events, sweeps) against
the oracle, bit for bit, in every sweep form, record mode, batch, shard and checkpoint path."""
import numpy as np
import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m.load()


def _metrics_array(g):
    d = g.metrics()
    return np.array([d["accepted"], d["tunnelling_events"], d["accepted_total"], d["tunnelling_events_total"],
                     d["sweeps"]], dtype=np.uint64)


def _run(system, L, q, p, seed, iters, sweeps, pipeline, record=0, beta=0.44, block=None):
    g = m.Muca(system, L, q, p, seed, beta=beta if system == m.ISING2D_MUMA else None, record=record, block=block)
    g.set_param("pipeline", pipeline)
    o = oracle.Run(system, L, q, p, seed, beta=beta if system == m.ISING2D_MUMA else 0.0, record=record)
    o.init()
    for it in range(iters):
        g.iterate(sweeps)
        g.merge_and_update()
        o.iterate(sweeps, 16)
        o.update()
        np.testing.assert_array_equal(_metrics_array(g), o.metrics(), err_msg="iteration %d" % it)
    compare_state(g, o, "after the metrics run")
    return g, o


@pytest.mark.parametrize("pipeline", [0, 1, 2])
@pytest.mark.parametrize("system,L,q,p", [(m.ISING2D, 8, 2, 96), (m.POTTS2D, 8, 3, 96), (m.ISING2D_MUMA, 8, 2, 96)])
def test_metrics_bit_exact(system, L, q, p, pipeline):
    g, o = _run(system, L, q, p, 7, 14, 150, pipeline)
    assert o.metrics()[3] > 0, "no tunnelling event in the run: the count was not exercised"


@pytest.mark.parametrize("pipeline", [0, 1])
def test_metrics_tiny_lattice_and_record_per_sweep(pipeline):
    _run(m.ISING2D, 4, 2, 40, 3, 8, 100, pipeline, record=1)
    _run(m.POTTS2D, 4, 4, 40, 3, 8, 100, pipeline)


def test_metrics_potts_code_form_large():
    """Potts q = 10, L = 48 in the code form (three producer parts, two-row ring): accepted
    counts of two iterations."""
    _run(m.POTTS2D, 48, 10, 64, 5, 2, 6, 2, block=32)


def test_metrics_batch_equals_individual_runs():
    mix = [(m.ISING2D, 8, 2, 64, 1, None), (m.POTTS2D, 8, 4, 64, 2, None), (m.ISING2D_MUMA, 8, 2, 64, 3, 0.44)]
    ref = [m.Muca(s, L, q, p, seed, beta=b) for s, L, q, p, seed, b in mix]
    for _ in range(4):
        for c in ref:
            c.iterate(40)
            c.merge_and_update()
    sys_ = [m.Muca(s, L, q, p, seed, beta=b) for s, L, q, p, seed, b in mix]
    bt = m.Batch(sys_)
    bt.run(2, 40, use_graph=False)
    bt.run(2, 40, use_graph=True)
    for r, s in zip(ref, sys_):
        assert r.metrics() == s.metrics()
    bt.close()


def test_metrics_of_shards_add_up():
    """Shards of one system (walker_offset) count their own walkers: in the first iteration (all
    contexts on the same weights) their counts add up to those of one context."""
    f0 = m.Muca(m.ISING2D, 8, 2, 100, 9)
    a0 = m.Muca(m.ISING2D, 8, 2, 37, 9)
    a1 = m.Muca(m.ISING2D, 8, 2, 63, 9, walker_offset=37)
    for c in (f0, a0, a1):
        c.iterate(50)
        c.merge_and_update()
    mf, m0, m1 = f0.metrics(), a0.metrics(), a1.metrics()
    assert mf["accepted"] == m0["accepted"] + m1["accepted"]
    assert mf["tunnelling_events"] == m0["tunnelling_events"] + m1["tunnelling_events"]
    assert mf["sweeps"] == m0["sweeps"] == m1["sweeps"] == 50


def test_metrics_survive_checkpoint():
    a = m.Muca(m.ISING2D, 8, 2, 64, 21)
    for _ in range(5):
        a.iterate(60)
        a.merge_and_update()
    b = m.Muca(m.ISING2D, 8, 2, 64, 21)
    for _ in range(3):
        b.iterate(60)
        b.merge_and_update()
    b.iterate(25)  # open iteration: its counts are part of the state
    c = m.Muca(m.ISING2D, 8, 2, 64, 21)
    c.set_state(b.get_state())
    c.iterate(35)
    c.merge_and_update()
    c.iterate(60)
    c.merge_and_update()
    assert a.metrics() == c.metrics()


def test_polymer_metrics_first_iteration_exact():
    """Wide window, ln W = 0: both sides accept exactly the moves that keep the bonds intact
    (the trajectories are bit-identical), so the accepted counts agree exactly."""
    N, p, S = 13, 48, 40
    g = m.Muca(m.POLYMER3D, N, 0, p, 5, window=(0.0, 1000.0))
    o = oracle.PolyRun(N, p, 5, 0.0, 1000.0)
    o.init()
    g.iterate(S)
    g.merge_and_update()
    o.iterate(S, 8)
    o.update()
    np.testing.assert_array_equal(g.coords(), o.coords())
    np.testing.assert_array_equal(_metrics_array(g), o.metrics())
    assert g.metrics()["acceptance_rate"] > 0.5


def test_jsonl_log_of_a_run(tmp_path):
    from paper_1312_2213_gb300.log import JsonlLog
    import json

    g = m.Muca(m.ISING2D, 8, 2, 64, 4)
    o = oracle.Run(m.ISING2D, 8, 2, 64, 4)
    o.init()
    path = str(tmp_path / "run.jsonl")
    with JsonlLog(path) as log:
        for it in range(3):
            g.iterate(30)
            g.merge_and_update()
            o.iterate(30, 8)
            o.update()
            log.log(g, seconds=1.0)
    recs = [json.loads(x) for x in open(path)]
    assert [r["iteration"] for r in recs] == [1, 2, 3]
    om = o.metrics()
    assert recs[-1]["accepted"] == int(om[0]) and recs[-1]["tunnelling_events"] == int(om[1])
    assert recs[-1]["bins_visited"] == int(np.count_nonzero(o.histogram()))
    assert recs[0]["acceptance_rate"] == 1.0  # ln W = 0: every move accepted
