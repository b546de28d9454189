"""Statistical speedup of the parallel scheme on one GPU.

For a degree of parallelisation p the weights start at ln W = 0 and every iteration runs
M_opt(L, p) sweeps per walker (Eq. 4 fits; the Ising fit is used for the multimagnetic
system as well, since the paper extrapolates it to its other spin systems); the run has
converged at the first iteration whose merged histogram is flat (every reachable bin
visited and min >= ratio * mean).  The mean over independent seeds, N_iter(p), gives the
time-independent speedup of Eq. 6,

    S*_p = [N_iter M_opt(1)]_1 / [N_iter M_opt(p)]_p,

with the sweep counts actually run (M_opt rounded, at least one sweep).  All seeds of one p
advance together in one batched launch per iteration.

    python -m paper_1312_2213_gb300.speedup --system ising --L 16 --p 1,4,16,64,256,1024,4096 --seeds 16
"""
from __future__ import annotations

import argparse
import json
import math
import sys
import time

import numpy as np

from . import ISING2D, ISING2D_MUMA, POTTS2D, Batch, Muca

SYSTEMS = {"ising": ISING2D, "potts": POTTS2D, "muma": ISING2D_MUMA}


def m_opt(system: int, L: int, p: int, q: int = 8) -> int:
    """Sweeps per iteration per walker, Eq. 4 (Ising fit for Ising and MUMA, 8-state Potts fit
    for Potts), rounded, at least one."""
    if system == POTTS2D:
        m = 24.0 * L ** 2.67 / p
    else:
        m = 5.7 * L ** 2.51 / p
    return max(1, int(round(m)))


def iterations_to_flat(system: int, L: int, q: int, p: int, seeds, sweeps: int, max_iter: int,
                       ratio: float = 0.5, beta: float | None = None):
    """Iterations until the first flat merged histogram, one entry per seed (None: not within
    max_iter).  All seeds advance together in one batch."""
    systems = [Muca(system, L, q, p, int(s), beta=beta) for s in seeds]
    for c in systems:
        c.set_param("flat_ratio", ratio)
    batch = Batch(systems)
    n_iter: list[int | None] = [None] * len(systems)
    try:
        for it in range(1, max_iter + 1):
            batch.run(1, sweeps, use_graph=False)
            for k, c in enumerate(systems):
                if n_iter[k] is None:
                    mn, mean, _ = c.flatness()
                    if mn > 0 and mn >= ratio * mean:
                        n_iter[k] = it
            if all(n is not None for n in n_iter):
                break
    finally:
        batch.close()
        for c in systems:
            c.close()
    return n_iter


def study(system: int, L: int, q: int, p_values, n_seeds: int, max_iter: int, ratio: float = 0.5,
          beta: float | None = None, seed0: int = 1000, log=None):
    rows = []
    for p in p_values:
        M = m_opt(system, L, p, q)
        t0 = time.perf_counter()
        seeds = [seed0 + 7919 * k + p for k in range(n_seeds)]
        n = iterations_to_flat(system, L, q, p, seeds, M, max_iter, ratio, beta)
        done = [x for x in n if x is not None]
        row = {"p": p, "sweeps_per_iteration": M, "seeds": n_seeds, "converged": len(done),
               "n_iter_mean": float(np.mean(done)) if done else math.nan,
               "n_iter_err": float(np.std(done, ddof=1) / math.sqrt(len(done))) if len(done) > 1 else math.nan,
               "seconds": time.perf_counter() - t0}
        rows.append(row)
        if log:
            log(row)
    base = next((r for r in rows if r["p"] == 1 and r["converged"]), None)
    # without p = 1 (a single chain can take too long), S* relative to the smallest converged p:
    # p0 S*_p / S*_p0 = p0 [N_iter M]_p0 / [N_iter M]_p, which equals S*_p where S*_p0 = p0
    ref = next((r for r in sorted(rows, key=lambda r: r["p"]) if r["converged"]), None)
    for r in rows:
        if base and r["converged"]:
            r["S_star"] = base["n_iter_mean"] * base["sweeps_per_iteration"] / (
                r["n_iter_mean"] * r["sweeps_per_iteration"])
        else:
            r["S_star"] = math.nan
        if ref and r["converged"]:
            r["S_star_rel"] = ref["p"] * ref["n_iter_mean"] * ref["sweeps_per_iteration"] / (
                r["n_iter_mean"] * r["sweeps_per_iteration"])
            r["S_star_rel_to_p"] = ref["p"]
        else:
            r["S_star_rel"] = math.nan
    return rows


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--system", choices=sorted(SYSTEMS), default="ising")
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--q", type=int, default=8)
    ap.add_argument("--beta", type=float, default=0.4407, help="multimagnetic inverse temperature")
    ap.add_argument("--p", default="1,2,4,8,16,32,64,128,256,512,1024,2048,4096,8192")
    ap.add_argument("--seeds", type=int, default=16)
    ap.add_argument("--max-iter", type=int, default=2000)
    ap.add_argument("--ratio", type=float, default=0.5)
    args = ap.parse_args(argv)
    system = SYSTEMS[args.system]
    q = args.q if system == POTTS2D else 2
    p_values = [int(x) for x in args.p.split(",")]
    beta = args.beta if system == ISING2D_MUMA else None
    rows = study(system, args.L, q, p_values, args.seeds, args.max_iter, args.ratio, beta,
                 log=lambda r: print(json.dumps({"partial": r}), file=sys.stderr, flush=True))
    for r in rows:
        print(json.dumps({"system": args.system, "L": args.L, "q": q, **r}), flush=True)


if __name__ == "__main__":
    main()
