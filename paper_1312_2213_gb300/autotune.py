"""Launch-shape autotuner.

For a lattice system the sweep form (`pipeline`: code form, producer/consumer, one warp) and the
walkers per thread block (`block`) change how fast a sweep runs but never what it computes: every
combination gives bit-identical lattices, histograms and weights.  For the polymer the same holds
for the threads per block (the lanes per walker do change the FP32 rounding, so they are left as
set).  The tuner times each valid combination on a scratch context of the same system, size and
walker count (a short iterate after a warm-up, CUDA events), keeps the fastest, and caches the
choice per (system, size, q, walkers, GPU) in a JSON file, `$MUCA_TUNE_CACHE` or
`~/.cache/muca_autotune.json`.

    from paper_1312_2213_gb300 import Muca, ISING2D, autotune
    g = Muca(ISING2D, 32, 2, 8192, seed)
    autotune.apply(g)          # before the first iterate
"""
from __future__ import annotations

import json
import os

from . import ISING2D_MUMA, POLYMER3D, Muca

SPIN_CANDIDATES = [(2, 32), (2, 64), (1, 32), (1, 64), (1, 128), (1, 256), (0, 64), (0, 128), (0, 256)]
POLY_CANDIDATES = [128, 256, 512]


def cache_path() -> str:
    return os.environ.get("MUCA_TUNE_CACHE") or os.path.join(os.path.expanduser("~"), ".cache", "muca_autotune.json")


def _key(system, L, q, p, device):
    return "%d/%d/%d/%d/%s" % (system, L, q, p, device)


def _device_name() -> str:
    import torch

    return torch.cuda.get_device_name(0).replace("/", "_")


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path, data):
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(data, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def _time_spin(system, L, q, p, pipeline, block, sweeps, beta):
    import torch

    g = Muca(system, L, q, p, 12345, beta=beta if system == ISING2D_MUMA else None, block=block)
    try:
        g.set_param("pipeline", pipeline)
        g.iterate(max(1, sweeps // 4))
        g.merge_and_update()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.iterate(sweeps)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    finally:
        g.close()


def _time_poly(N, p, block, sweeps, window):
    import torch

    g = Muca(POLYMER3D, N, 0, p, 12345, window=window, block=block)
    try:
        g.iterate(max(1, sweeps // 4))
        g.merge_and_update()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.iterate(sweeps)
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b)
    finally:
        g.close()


def tune(system: int, L: int, q: int, p: int, beta: float = 0.4407, window=None, sweeps: int | None = None,
         use_cache: bool = True, timer=None) -> dict:
    """Fastest launch shape for the configuration: {"pipeline", "block", "ms", "timings"} for lattice
    systems, {"block", "ms", "timings"} for the polymer.  `timer` replaces the CUDA-event timing
    (for tests)."""
    path = cache_path()
    device = _device_name() if timer is None else "test"
    key = _key(system, L, q, p, device)
    data = _load(path) if use_cache else {}
    if use_cache and key in data:
        return data[key]
    timings = {}
    if system == POLYMER3D:
        sw = sweeps or max(2, int(2e7 / (p * L)))
        for block in POLY_CANDIDATES:
            t = (timer or (lambda b: _time_poly(L, p, b, sw, window)))(block)
            if t is not None:
                timings[str(block)] = t
        best = min(timings, key=timings.get)
        res = {"block": int(best), "ms": timings[best], "timings": timings}
    else:
        sw = sweeps or max(2, int(4e8 / (p * L * L)))
        for pipeline, block in SPIN_CANDIDATES:
            if block > p and block != 32:
                continue
            try:
                t = (timer or (lambda pl, bl: _time_spin(system, L, q, p, pl, bl, sw, beta)))(pipeline, block)
            except Exception:
                t = None  # a shape this configuration cannot run
            if t is not None:
                timings["%d/%d" % (pipeline, block)] = t
        best = min(timings, key=timings.get)
        pl, bl = (int(x) for x in best.split("/"))
        res = {"pipeline": pl, "block": bl, "ms": timings[best], "timings": timings}
    if use_cache:
        data = _load(path)
        data[key] = res
        _store(path, data)
    return res


BATCH_BLOCKS = (32, 64)  # walkers per block of the code form


def _weight(spec) -> float:
    system, L = spec[0], spec[1]
    return L if system == POLYMER3D else L * L * (2.5 if system == 1 else 1.0)


MIN_GAIN = 0.03  # a batch shape must shorten the iteration by this much to replace another


def _time_batch(specs, blocks, sweeps, iters=3):
    """Milliseconds of one graph-captured batch iteration (the best of `iters`) on scratch
    contexts with the given walkers per block (None: the context's default)."""
    import torch

    from . import Batch

    ctxs = []
    try:
        for k, (system, L, q, p, extra) in enumerate(specs):
            kw = {"block": blocks[k]} if blocks[k] is not None else {}
            if system == POLYMER3D:
                kw["window"] = extra
            elif system == ISING2D_MUMA:
                kw["beta"] = extra
            ctxs.append(Muca(system, L, q, p, 777 + k, **kw))
        b = Batch(ctxs)
        try:
            b.set_sweeps(sweeps)
            b.run(1, 1, use_graph=True)  # capture and warm up
            best = None
            for _ in range(iters):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                b.run(1, 1, use_graph=True)
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1)
                best = t if best is None else min(best, t)
            return best
        finally:
            b.close()
    finally:
        for c in ctxs:
            c.close()


def tune_batch(specs, sweeps, timer=None, use_cache: bool = True) -> dict:
    """Walkers per block for every lattice system of a side-by-side batch, chosen on the batch's
    own iteration time: the systems share the SMs, so the best shape of a system alone need not be
    the best inside the batch.  `specs` lists (system, L, q, p, extra) with extra = beta for the
    multimagnetic system, the window for a polymer, else None; `sweeps` the sweeps of each system
    an iteration (as for Batch.set_sweeps).  Coordinate descent from the library's defaults: for
    every lattice system, heaviest first, each other block size of the code form is timed with the
    rest fixed and kept if the iteration gets shorter by at least MIN_GAIN (the spread of one
    batch timing is a few per cent: where the blocks of nine systems land varies).  Polymers keep their block.  Returns
    {"blocks": [...] (None = the default), "ms": ..., "trials": n}; `timer(blocks)` replaces the
    timing (tests)."""
    specs = [tuple(s_) for s_ in specs]
    sweeps = [int(x) for x in sweeps]
    path = cache_path()
    device = _device_name() if timer is None else "test"
    key = "batch/%s/%s/%s" % (json.dumps(specs), json.dumps(sweeps), device)
    data = _load(path) if use_cache else {}
    if use_cache and key in data:
        return data[key]
    t_of = timer or (lambda blocks: _time_batch(specs, blocks, sweeps))
    blocks = [None] * len(specs)
    best = t_of(blocks)
    trials = 1
    order = sorted(range(len(specs)), key=lambda k: -_weight(specs[k]) * sweeps[k])
    for k in order:
        if specs[k][0] == POLYMER3D:
            continue
        for cand in BATCH_BLOCKS:
            trial = list(blocks)
            trial[k] = cand
            try:
                t = t_of(trial)
            except Exception:
                t = None  # a block size this system's code form cannot take
            trials += 1
            if t is not None and t < best * (1.0 - MIN_GAIN):
                best, blocks = t, trial
    res = {"blocks": blocks, "ms": best, "trials": trials}
    if use_cache:
        data = _load(path)
        data[key] = res
        _store(path, data)
    return res


def apply_batch(contexts, sweeps, **kw) -> dict:
    """Tune the walkers per block of the contexts for a batch with these per-system sweeps and set
    them; call before the contexts' first iterate and before creating the Batch."""
    specs = []
    for g in contexts:
        extra = g.window if g.system == POLYMER3D else (g.beta if g.system == ISING2D_MUMA else None)
        specs.append((g.system, g.L, g.q, g.p, extra))
    res = tune_batch(specs, sweeps, **kw)
    for g, bl in zip(contexts, res["blocks"]):
        if bl is not None:
            g.set_param("block", bl)
    return res


def apply(g: Muca, **kw) -> dict:
    """Tune (or look up) the context's configuration and set the result on it; call before its
    first iterate."""
    res = tune(g.system, g.L, g.q, g.p, window=g.window, **kw)
    g.set_param("block", res["block"])
    if g.system != POLYMER3D:
        g.set_param("pipeline", res["pipeline"])
    return res
