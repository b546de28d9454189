"""The launch-shape autotuner on the GPU: it times real shapes, returns a valid choice, and a
context set to that choice stays bit-exact against the oracle (no shape changes results)."""
import pytest

import oracle
import paper_1312_2213_gb300 as m
from gpu_util import compare_state
from paper_1312_2213_gb300 import autotune

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    import torch

    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_tuned_context_stays_bit_exact(tmp_path, monkeypatch):
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    r = autotune.tune(m.ISING2D, 16, 2, 256, sweeps=40)
    assert r["block"] in (32, 64, 128, 256) and r["pipeline"] in (0, 1, 2) and len(r["timings"]) >= 6
    g = m.Muca(m.ISING2D, 16, 2, 256, 77)
    autotune.apply(g)   # from the cache written above
    o = oracle.Run(0, 16, 2, 256, 77)
    o.init()
    for _ in range(3):
        g.iterate(12)
        g.merge_and_update()
        o.iterate(12, 8)
        o.update()
    compare_state(g, o, "after autotuning")


def test_polymer_block_tuning(tmp_path, monkeypatch):
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    r = autotune.tune(m.POLYMER3D, 13, 0, 512, window=(33.3, 87.3), sweeps=4)
    assert r["block"] in autotune.POLY_CANDIDATES


def test_batch_tuning_keeps_results(tmp_path, monkeypatch):
    """The batch tuner times real batch iterations, returns a code-form block (or the default) for
    every lattice system, and contexts set to its choice give the same results as default ones."""
    import numpy as np

    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    spec = [(m.ISING2D, 32, 2, 300, None), (m.POTTS2D, 16, 10, 200, None), (m.ISING2D_MUMA, 16, 2, 100, 0.4407)]
    sweeps = [6, 9, 4]
    r = autotune.tune_batch(spec, sweeps)
    assert len(r["blocks"]) == 3 and all(b in (None, 32, 64) for b in r["blocks"]) and r["trials"] == 7
    runs = []
    for tuned in (False, True):
        ctx = [m.Muca(s_, L, q, p, 90 + k, beta=x) for k, (s_, L, q, p, x) in enumerate(spec)]
        if tuned:
            autotune.apply_batch(ctx, sweeps)  # from the cache written above
        b = m.Batch(ctx)
        b.set_sweeps(sweeps)
        b.run(3, 1)
        runs.append([(c.histogram(), c.spins(), c.lnW().view(np.uint64)) for c in ctx])
        b.close()
    for x, y in zip(*runs):
        for a_, b_ in zip(x, y):
            np.testing.assert_array_equal(a_, b_)
