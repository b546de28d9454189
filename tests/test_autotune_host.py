"""Host logic of the launch-shape autotuner: picks the fastest valid shape, skips shapes that fail,
caches per configuration."""
import json

import paper_1312_2213_gb300 as m
from paper_1312_2213_gb300 import autotune


def test_picks_fastest_and_caches(tmp_path, monkeypatch):
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    calls = []

    def timer(pipeline, block):
        calls.append((pipeline, block))
        if (pipeline, block) == (1, 256):
            raise RuntimeError("does not fit")
        return {(2, 64): 1.0, (2, 32): 1.5}.get((pipeline, block), 3.0)

    r = autotune.tune(m.ISING2D, 32, 2, 8192, timer=timer)
    assert (r["pipeline"], r["block"]) == (2, 64)
    assert "1/256" not in r["timings"]
    n = len(calls)
    r2 = autotune.tune(m.ISING2D, 32, 2, 8192, timer=timer)  # from the cache: no timing
    assert r2 == r and len(calls) == n
    data = json.load(open(tmp_path / "tune.json"))
    assert len(data) == 1


def test_small_walker_counts_skip_large_blocks(tmp_path, monkeypatch):
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    seen = []
    autotune.tune(m.POTTS2D, 16, 5, 40, timer=lambda pl, bl: seen.append(bl) or float(bl), use_cache=False)
    assert max(seen) <= 64


def test_polymer_tunes_block_only(tmp_path, monkeypatch):
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    r = autotune.tune(m.POLYMER3D, 32, 0, 4096, timer=lambda b: {128: 2.0, 256: 1.0, 512: 1.5}[b])
    assert r["block"] == 256 and "pipeline" not in r
