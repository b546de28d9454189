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


def test_batch_tuner_descends_per_system(tmp_path, monkeypatch):
    """The batch tuner starts from the defaults and keeps a block size only where the whole
    batch's iteration gets shorter; polymers are left alone; the result is cached."""
    monkeypatch.setenv("MUCA_TUNE_CACHE", str(tmp_path / "tune.json"))
    specs = [(m.ISING2D, 64, 2, 2048, None), (m.POTTS2D, 32, 10, 2048, None),
             (m.POLYMER3D, 13, 0, 1024, (33.3, 87.3)), (m.ISING2D_MUMA, 16, 2, 512, 0.4407)]
    seen = []

    def timer(blocks):  # the Potts system prefers 64 inside this batch, Ising L = 64 its default
        seen.append(tuple(blocks))
        t = 10.0
        if blocks[1] == 64:
            t -= 2.0
        if blocks[0] == 32:
            t += 5.0
        if blocks[3] == 32:
            raise RuntimeError("does not fit")
        return t

    r = autotune.tune_batch(specs, [95, 122, 150, 3], timer=timer)
    assert r["blocks"] == [None, 64, None, None] and r["ms"] == 8.0
    assert all(b[2] is None for b in seen)  # the polymer's block is never tried
    n = len(seen)
    assert autotune.tune_batch(specs, [95, 122, 150, 3], timer=timer) == r and len(seen) == n
