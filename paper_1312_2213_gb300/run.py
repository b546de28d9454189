"""Run a multicanonical simulation from a JSON configuration (the files under configs/).

    python -m paper_1312_2213_gb300.run configs/ising2d_L8_p64.json --log run.jsonl

A configuration names one system or a list of them ("systems"; several lattice systems are
advanced together as a batch, in one CUDA graph per iteration when "graph" is true; polymers run
one after the other):

    {"systems": [{"system": "ising2d", "L": 32, "q": 2, "p": 8192, "seed": 1}],
     "iterations": 30, "sweeps": 10000, "stop_when_flat": false, "flat_ratio": 0.5,
     "reweight_betas": [0.3, 0.4407]}

Per system: "system" (ising2d, potts2d, ising2d_muma, polymer3d), "L" (beads N for the polymer),
"q", "p", "seed", and optionally "beta" (multimagnetic), "window" ([e_lo, e_hi] for the polymer,
or "pilot" for the packaged pilot window of that N), "record", "block", "pipeline", "model",
"moves", "recursion", "observables".  Each closed iteration appends one JSON line per system to
the log (paper_1312_2213_gb300.log); the last line printed holds the final flatness and, for every
beta in "reweight_betas", the Eq. 2 reweighting of the last merged histogram.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

from . import POLYMER3D, SYSTEM_NAMES, Batch, Muca
from .log import JsonlLog

SYSTEMS = {v: k for k, v in SYSTEM_NAMES.items()}
_PARAMS = ("pipeline", "model", "moves", "recursion", "observables", "flat_ratio")


def _pilot_window(N: int):
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "polymer_windows.json")
    with open(path) as f:
        w = json.load(f)["windows"][str(N)]
    return (w["e_lo"], w["e_hi"])


def make_system(spec: dict, flat_ratio: float = 0.5) -> Muca:
    system = SYSTEMS[spec["system"]]
    window = spec.get("window")
    if window == "pilot":
        window = _pilot_window(spec["L"])
    c = Muca(system, spec["L"], spec.get("q", 2), spec["p"], spec.get("seed", 1), beta=spec.get("beta"),
             record=spec.get("record", 0), block=spec.get("block"),
             window=tuple(window) if window is not None else None)
    c.set_param("flat_ratio", spec.get("flat_ratio", flat_ratio))
    for k in _PARAMS[:-1]:
        if k in spec:
            c.set_param(k, spec[k])
    return c


def _flat(c, ratio: float) -> bool:
    mn, mean, _ = c.flatness()
    return bool(mn > 0 and mn >= ratio * mean)


def run(cfg: dict, log=None, out=sys.stdout) -> dict:
    specs = cfg["systems"] if "systems" in cfg else [cfg]
    ratio = cfg.get("flat_ratio", 0.5)
    systems = [make_system(s, ratio) for s in specs]
    ratios = [s.get("flat_ratio", ratio) for s in specs]
    iters, sweeps = int(cfg.get("iterations", 10)), int(cfg.get("sweeps", 1000))
    stop = bool(cfg.get("stop_when_flat", False))
    spins_only = all(c.system != POLYMER3D for c in systems)
    batch = Batch(systems) if len(systems) > 1 and spins_only else None
    graph = bool(cfg.get("graph", False)) and batch is not None
    done = 0
    try:
        for it in range(iters):
            t0 = time.perf_counter()
            if batch is not None:
                batch.run(1, sweeps, use_graph=graph)
            else:  # one system, or polymers (not part of spin batches): one after the other
                for c in systems:
                    c.iterate(sweeps)
                    c.merge_and_update()
            for c in systems:
                c.synchronize()
            dt = time.perf_counter() - t0
            done = it + 1
            if log is not None:
                for c in systems:
                    log.log(c, seconds=dt / len(systems))
            if stop and all(_flat(c, r) for c, r in zip(systems, ratios)):
                break
        result = {"iterations": done, "systems": []}
        for c, s, ratio_c in zip(systems, specs, ratios):
            mn, mean, mx = (float(x) for x in c.flatness())
            r = {"system": s["system"], ("N" if c.system == POLYMER3D else "L"): c.L, "p": c.p,
                 "flat": _flat(c, ratio_c), "h_min": mn, "h_mean": mean, "h_max": mx, "reweight": {}}
            for beta in cfg.get("reweight_betas", []):
                vals, _ = c.reweight(float(beta))
                r["reweight"][str(beta)] = [float(v) for v in vals]
            result["systems"].append(r)
        print(json.dumps(result), file=out, flush=True)
        return result
    finally:
        if batch is not None:
            batch.close()
        for c in systems:
            c.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("config")
    ap.add_argument("--log", help="append one JSON line per system and iteration to this file")
    ap.add_argument("--iterations", type=int, help="override the configuration's iteration count")
    ap.add_argument("--sweeps", type=int, help="override the configuration's sweeps per iteration")
    args = ap.parse_args(argv)
    with open(args.config) as f:
        cfg = json.load(f)
    if args.iterations:
        cfg["iterations"] = args.iterations
    if args.sweeps:
        cfg["sweeps"] = args.sweeps
    log = JsonlLog(args.log) if args.log else None
    try:
        run(cfg, log)
    finally:
        if log is not None:
            log.close()


if __name__ == "__main__":
    main()
