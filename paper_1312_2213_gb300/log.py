"""Per-iteration metrics of a multicanonical run as JSON lines.

After each merge_and_update, `JsonlLog.log(ctx)` appends one line: the closed iteration's index and
sweeps, its accepted moves and acceptance rate, its tunnelling events (and the running total), the
flatness of its merged histogram over the reachable bins (H_min, H_mean, H_max and their ratios),
the number of reachable bins it visited and, when the caller passes the iteration's wall time,
attempts/s.

    log = JsonlLog("run.jsonl")
    for it in range(n):
        t0 = time.perf_counter(); g.iterate(M); g.merge_and_update(); g.synchronize()
        log.log(g, seconds=time.perf_counter() - t0)
"""
from __future__ import annotations

import json
import math

import numpy as np

from . import POLYMER3D, SYSTEM_NAMES


def record(ctx, seconds: float | None = None, **extra) -> dict:
    """The metrics of the context's last closed iteration as a dict."""
    met = ctx.metrics()
    H = ctx.histogram().astype(np.float64)
    reach = np.isfinite(ctx.lnW())
    h = H[reach]
    h_min, h_mean, h_max = (float(h.min()), float(h.mean()), float(h.max())) if h.size else (0.0, 0.0, 0.0)
    rec = {"system": SYSTEM_NAMES[ctx.system], ("N" if ctx.system == POLYMER3D else "L"): ctx.L,
           "q": ctx.q, "p": ctx.p}
    rec.update(met)
    rec.update({"h_min": h_min, "h_mean": h_mean, "h_max": h_max,
                "h_min_over_mean": h_min / h_mean if h_mean > 0 else math.nan,
                "h_min_over_max": h_min / h_max if h_max > 0 else math.nan,
                "bins_visited": int(np.count_nonzero(h)), "bins_reachable": int(h.size)})
    if seconds is not None and seconds > 0:
        rec["seconds"] = seconds
        rec["attempts_per_s"] = ctx.p * ctx.N * met["sweeps"] / seconds
    rec.update(extra)
    return rec


class JsonlLog:
    def __init__(self, path_or_file):
        self._own = isinstance(path_or_file, str)
        self.f = open(path_or_file, "a") if self._own else path_or_file

    def log(self, ctx, seconds: float | None = None, **extra) -> dict:
        rec = record(ctx, seconds, **extra)
        self.f.write(json.dumps(rec) + "\n")
        self.f.flush()
        return rec

    def close(self):
        if self._own:
            self.f.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
