#!/usr/bin/env python
"""Benchmark of the parallel multicanonical hot path on GB300.

Workload (one "step" = one multicanonical iteration of the Fig. 1 loop for each system):
  * 2D Ising L = 32, periodic, p = 8192 walkers, multicanonical in E (bins E = -2048..2048 step 4);
  * 2D Ising L = 32, p = 8192, multimagnetic in M at beta = 0.4407 (Eq. 3);
each with 1e4 sweeps of every walker, then the histogram merge, the accumulated-statistics
recursion of ln W and the threshold rebuild.  Metric: move attempts per second (an attempt is one
proposed single-spin update, accepted or not), whole job.

  value      device-timed (CUDA events on the launching stream), state resident in HBM;
  e2e        the same step through the C ABI with the state copied in from pinned host memory
             (muca_set_state) and back out (muca_get_state) every step;
  roofline   the sweep kernel against the integer issue peak (SMs x 4 schedulers x 32 lanes x f_SM);
  cpu_baseline  the CPU oracle (all host cores) on a bounded sample of the same workload.
  batched_mix   the uneven mix (2D Ising L in {16,24,32,48,64} and q=10 Potts L in {16,24,32,48},
                2048 walkers each): one system per launch (plain) against all systems in one
                persistent launch per iteration, and against the whole loop as one CUDA graph.
  polymer       the bead-spring polymer, N in {13,32,64,128}, p = 4096, in its pilot windows.

With N > 1 GPUs (torchrun) each system's walkers are split over the ranks (8192 a rank, weak
scaling) and every iteration ends with one all-reduce of the B-bin histogram per system (the
paper's Fig. 1 exchange, NCCL on device buffers) before the identical recursion on every rank;
`--mode replicas` runs an independent system pair per rank instead.

`--impl reference` times the CPU oracle itself as the reference arm.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L, P, SWEEPS, BETA_MUMA = 32, 8192, 10000, 0.4407
N = L * L
# Algorithmic integer instructions per attempt of the spin sweep (per walker-thread); the
# breakdown is stated with the kernel: Philox4x32-10 amortised over the 4 words of one call
# (10 rounds x 4 ops / 4 = 10), neighbour bits and count 8, table column and address 2,
# threshold load 1, integer compare 2, flip/select 3, bin update 2, histogram atomic 1, loop 1.
INSTR_PER_ATTEMPT = 30
# Cycles an attempt of one walker's chain in this design's sweep with its scheduler to itself
# (one consumer warp an SM, p = 4096 in 32-walker blocks, measured on GB300 at 2.07 GHz): Ising
# 42.9, multimagnetic 49.1, averaged over the step's two systems.  p f / CHAIN_CYCLES bounds the
# attempts/s of the sweep kernel, and its rate is reported against it as well (the issue-peak
# fraction counts all schedulers, which one chain per walker cannot fill at p = 8192).
CHAIN_CYCLES = (42.9 + 49.1) / 2
# DRAM bytes (read + write) per launch of the timed sweep kernel, from one ncu capture of the current
# k_sweep_spin_tn build (dram__bytes_read.sum + dram__bytes_write.sum; mean of the Ising and MUMA
# launches: 1.25 MB and 2.17 MB read, nothing written).  It is the walker state and does not grow
# with the sweep count.  Set to None whenever the kernel changes until it is measured again.
TRAFFIC_PER_LAUNCH = 1.71e6
# The headline metric as the benchmark specification names it; the workload it is quoted on here
# (2D Ising L = 32, p = 8192: MUCA in E plus the multimagnetic run) is in the line's "config".
METRIC = "MUCA move attempts/s on 1 GB300 (batched vs plain) + fraction of issue roofline"
UNIT = "attempts/s"
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--sweeps", type=int, default=SWEEPS)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sweeps", type=int, default=400, help="sweeps per system in the CPU sample")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched-mix, Potts and polymer measurements")
    ap.add_argument("--workload", default="all", choices=["all", "mix", "polymer", "potts", "potts64"],
                    help="mix / polymer / potts: run only that measurement (for profiling)")
    ap.add_argument("--mode", default="shard", choices=["shard", "replicas"],
                    help="N > 1: 'shard' runs each system's walkers split over the ranks with one histogram "
                         "all-reduce per iteration (Fig. 1); 'replicas' runs an independent system pair per rank")
    return ap.parse_args()


def make_sharded_systems(m, rank: int, world: int, stream=None, p_per_rank: int = P, ctx_factory=None,
                         device: str = "cuda"):
    """The workload split over `world` ranks with weak scaling: each system has p_per_rank walkers
    per rank (p_per_rank * world in all, one seed per system), rank r holding walkers
    [r p_per_rank, (r + 1) p_per_rank).  After every iteration's sweeps the ranks add their open
    histograms with one all-reduce of B uint64 per system and run the same recursion."""
    from paper_1312_2213_gb300.shard import ShardedMuca

    p_all = p_per_rank * world
    return [ShardedMuca(m.ISING2D if m else 0, L, 2, p_all, 1, ctx_factory=ctx_factory, device=device, stream=stream),
            ShardedMuca(m.ISING2D_MUMA if m else 2, L, 2, p_all, 1001, ctx_factory=ctx_factory, device=device,
                        beta=BETA_MUMA, stream=stream)]


def sharded_step(systems, sweeps: int, kevents=None, stream=None):
    """One step of the sharded workload: every system's sweeps on this rank's walkers, then the
    exchange and the update (kernel events around the sweeps if kevents is given)."""
    for s in systems:
        if kevents is not None:
            import torch

            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            s.iterate(sweeps)
            b.record(stream)
            kevents.append((a, b))
        else:
            s.iterate(sweeps)
        s.merge_and_update()


MIX = [(0, L, 2) for L in (16, 24, 32, 48, 64)] + [(1, L, 10) for L in (16, 24, 32, 48)]
MIX_P = 2048


def mix_mopt(p=MIX_P):
    """Each mix system's optimal iteration length from the fits of Eq. 4: M_opt = 5.7 L^2.51 / p
    (Ising) and 24 L^2.67 / p (the 8-Potts fit, used for q = 10)."""
    return [max(1, round((5.7 * L ** 2.51 if s_ == 0 else 24.0 * L ** 2.67) / p)) for s_, L, _ in MIX]


def run_mix(m, torch, sweeps=1000, short_sweeps=10, short_iters=20, mopt_iters=50):
    """Plain (one system per launch, host loop) vs batched (both batch forms) vs graph."""
    sites = sum(L * L for _, L, _ in MIX)

    def make(seed0):  # default walkers per block: the plain path runs the fastest form that fits
        return [m.Muca(s_, L, q, MIX_P, seed0 + i) for i, (s_, L, q) in enumerate(MIX)]

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    out = {"systems": "ising2d L=16,24,32,48,64 + potts2d q=10 L=16,24,32,48", "walkers_per_system": MIX_P}
    # throughput regime: 1 iteration of `sweeps` sweeps
    sysA = make(100)
    for c in sysA:       # warm-up iteration
        c.iterate(20)
        c.merge_and_update()

    def plain_iter(systems, sw):
        for c in systems:
            c.iterate(sw)
            c.merge_and_update()

    t_plain = timed(lambda: plain_iter(sysA, sweeps))
    t_plain_s = timed(lambda: [plain_iter(sysA, short_sweeps) for _ in range(short_iters)])
    mopt = mix_mopt()

    def plain_mopt():
        for c, sw in zip(sysA, mopt):
            c.iterate(sw)
            c.merge_and_update()

    t_plain_m = timed(lambda: [plain_mopt() for _ in range(mopt_iters)])
    att_m = MIX_P * sum(sw * L * L for sw, (_, L, _) in zip(mopt, MIX)) * mopt_iters
    att = MIX_P * sweeps * sites
    att_s = MIX_P * short_sweeps * sites * short_iters
    # batched forms: 0 = one persistent launch over all systems' tiles (one warp per 32 walkers),
    # 1 = every system's own (code-form) sweep kernel side by side on forked streams
    forms, made = {}, []
    for form in (0, 1):
        sysB = make(200 + 100 * form)
        made += sysB
        batch = m.Batch(sysB, form=form)
        batch.run(1, 20, use_graph=False)
        t_batch = timed(lambda: batch.run(1, sweeps, use_graph=False))
        batch.run(1, sweeps, use_graph=True)      # capture
        t_graph = timed(lambda: batch.run(1, sweeps, use_graph=True))
        batch.run(short_iters, short_sweeps, use_graph=True)  # capture
        t_graph_s = timed(lambda: batch.run(short_iters, short_sweeps, use_graph=True))
        t_batch_s = timed(lambda: batch.run(short_iters, short_sweeps, use_graph=False))
        batch.set_sweeps(mopt)  # every system at its own M_opt
        batch.run(mopt_iters, 1, use_graph=True)  # capture
        t_graph_m = timed(lambda: batch.run(mopt_iters, 1, use_graph=True))
        t_batch_m = timed(lambda: batch.run(mopt_iters, 1, use_graph=False))
        batch.close()
        forms[form] = (t_batch, t_graph, t_batch_s, t_graph_s, t_batch_m, t_graph_m)
    best = min(forms, key=lambda f: forms[f][1])
    t_batch, t_graph, t_batch_s, t_graph_s, t_batch_m, t_graph_m = forms[best]
    out["throughput"] = {"sweeps_per_iteration": sweeps, "attempts_per_iteration": att, "batch_form": best,
                         "plain_attempts_per_s": att / t_plain, "batched_attempts_per_s": att / t_batch,
                         "graph_attempts_per_s": att / t_graph, "batched_over_plain": t_plain / t_batch,
                         "graph_over_plain": t_plain / t_graph,
                         "by_form": {str(f): {"batched_attempts_per_s": att / v[0], "graph_attempts_per_s": att / v[1]}
                                     for f, v in forms.items()}}
    # short iterations: launch and host overheads dominate
    out["short_iterations"] = {"sweeps_per_iteration": short_sweeps, "iterations": short_iters, "batch_form": best,
                               "plain_attempts_per_s": att_s / t_plain_s, "batched_attempts_per_s": att_s / t_batch_s,
                               "graph_attempts_per_s": att_s / t_graph_s, "graph_over_plain": t_plain_s / t_graph_s,
                               "by_form": {str(f): {"batched_attempts_per_s": att_s / v[2],
                                                    "graph_attempts_per_s": att_s / v[3]} for f, v in forms.items()}}
    # each system at its own M_opt (Eq. 4) for p = 2048: uneven iteration lengths
    out["mopt_iterations"] = {"sweeps_per_iteration": dict(zip(["ising%d" % L if s_ == 0 else "potts%d" % L
                                                                for s_, L, _ in MIX], mopt)),
                              "iterations": mopt_iters, "batch_form": best,
                              "plain_attempts_per_s": att_m / t_plain_m, "batched_attempts_per_s": att_m / t_batch_m,
                              "graph_attempts_per_s": att_m / t_graph_m, "graph_over_plain": t_plain_m / t_graph_m,
                              "by_form": {str(f): {"batched_attempts_per_s": att_m / v[4],
                                                   "graph_attempts_per_s": att_m / v[5]} for f, v in forms.items()}}
    for c in sysA + made:
        c.close()
    return out


def run_potts(m, torch, L=32, q=8, p=8192, sweeps=2000):
    """Potts q = 8, L = 32, p = 8192 (the first-order Potts workload): one iteration of `sweeps` sweeps."""
    g = m.Muca(m.POTTS2D, L, q, p, 11)
    for _ in range(2):
        g.iterate(50)
        g.merge_and_update()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    g.iterate(sweeps)
    b.record()
    g.merge_and_update()
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    g.close()
    att = p * sweeps * L * L
    return {"L": L, "q": q, "walkers": p, "sweeps": sweeps, "attempts_per_s": att / t, "kernel_ms": t * 1e3}


def run_potts64(m, torch, q=10, sweeps=150):
    """q-Potts at L = 64 (the paper's Fig. 4 lattice; the code form with the split threshold table,
    64 walkers a block): p = 8192 and p = 9728 (one block on each of the 152 SMs)."""
    out = {"L": 64, "q": q, "sweeps": sweeps, "form": "code form, split threshold table"}
    for p in (8192, 9728):
        r = run_potts(m, torch, L=64, q=q, p=p, sweeps=sweeps)
        out["p%d" % p] = {"attempts_per_s": r["attempts_per_s"], "kernel_ms": r["kernel_ms"]}
    return out


def run_polymer(m, torch, p=4096, budget_attempts=2.0e8):
    import json as _json

    W = _json.load(open(os.path.join(ROOT, "paper_1312_2213_gb300", "polymer_windows.json")))["windows"]
    res = {"walkers": p, "windows": "pilot windows (paper_1312_2213_gb300/polymer_windows.json)", "chains": {}}
    for N in (13, 32, 64, 128):
        g = m.Muca(m.POLYMER3D, N, 0, p, 7, window=(W[str(N)]["e_lo"], W[str(N)]["e_hi"]))
        for _ in range(2):
            g.iterate(max(1, 200 // N))
            g.merge_and_update()
        sw = max(2, int(budget_attempts / (p * N)))
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        g.iterate(sw)
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b) / 1e3
        att = p * sw * N
        res["chains"][str(N)] = {"sweeps": sw, "attempts_per_s": att / t, "pair_evals_per_s": att * 2 * (N - 1) / t,
                                 "energy_drift": g.drift()}
        g.close()
    res["lengths_batched"] = run_polymer_batch(m, torch, W, p)
    return res


def run_polymer_batch(m, torch, W, p=4096, iters=3):
    """The four lengths side by side in one batch (each 2000 / N sweeps an iteration, so each does
    about the same attempts) against one after another (plain)."""
    Ns = (13, 32, 64, 128)
    sweeps = [max(1, 2000 // N) for N in Ns]

    def make(seed0):
        out = []
        for i, N in enumerate(Ns):
            g = m.Muca(m.POLYMER3D, N, 0, p, seed0 + i, window=(W[str(N)]["e_lo"], W[str(N)]["e_hi"]))
            g.iterate(max(1, 200 // N))
            g.merge_and_update()
            out.append(g)
        return out

    def timed(fn):
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    att = iters * p * sum(N * s_ for N, s_ in zip(Ns, sweeps))
    sysA = make(300)

    def plain():
        for _ in range(iters):
            for g, s_ in zip(sysA, sweeps):
                g.iterate(s_)
                g.merge_and_update()

    t_plain = timed(plain)
    sysB = make(400)
    batch = m.Batch(sysB)
    batch.set_sweeps(sweeps)
    batch.run(1, 1, use_graph=False)
    t_batch = timed(lambda: batch.run(iters, 1, use_graph=False))
    batch.run(iters, 1, use_graph=True)  # capture
    t_graph = timed(lambda: batch.run(iters, 1, use_graph=True))
    batch.close()
    for g in sysA + sysB:
        g.close()
    return {"sweeps_per_iteration": dict(zip([str(N) for N in Ns], sweeps)), "iterations": iters,
            "plain_attempts_per_s": att / t_plain, "batched_attempts_per_s": att / t_batch,
            "graph_attempts_per_s": att / t_graph, "graph_over_plain": t_plain / t_graph}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(sweeps: int, seed0: int):
    """The oracle, as it stands, over the same workload with fewer sweeps (all host cores)."""
    import oracle

    nth = os.cpu_count() or 1
    attempts = 0
    t0 = time.perf_counter()
    for system, beta, seed in ((oracle.ISING, 0.0, seed0), (oracle.MUMA, BETA_MUMA, seed0 + 1000)):
        r = oracle.Run(system, L, 2, P, seed, beta=beta)
        r.init()
        r.iterate(sweeps, nth)
        r.update()
        attempts += P * sweeps * N
    dt = time.perf_counter() - t0
    return {"value": attempts / dt, "unit": UNIT, "cores": nth, "kind": "oracle",
            "sample": "Ising L=32 p=8192 MUCA + MUMA, 1 iteration of %d sweeps each (%.3g attempts, %.1f s)"
                      % (sweeps, attempts, dt)}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle  # noqa: F401  (the reference arm is the CPU oracle)

    for _ in range(args.warmup):
        cpu_sample(max(1, args.cpu_sweeps // 10), 7)
    vals, tot_t = [], 0.0
    for k in range(args.steps):
        s = cpu_sample(args.cpu_sweeps, 7 + k)
        vals.append(s["value"])
    val = statistics.median(vals)
    step_attempts = 2 * P * args.cpu_sweeps * N
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_attempts / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": "ising2d_L32_p8192_muca+muma", "L": L, "p": P, "systems": 2,
                       "sweeps_per_step": args.cpu_sweeps, "note": "bounded sample of the 1e4-sweep step"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": "%d sweeps per system per step" % args.cpu_sweeps},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import paper_1312_2213_gb300 as m

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    m.load()
    stream = torch.cuda.Stream()
    sharded = world > 1 and args.mode == "shard"
    if sharded:
        systems = make_sharded_systems(m, rank, world, stream=stream)
        ctxs = [s.ctx for s in systems]
    else:
        seed = 1 + 7919 * rank
        systems = [m.Muca(m.ISING2D, L, 2, P, seed, stream=stream),
                   m.Muca(m.ISING2D_MUMA, L, 2, P, seed + 1000, beta=BETA_MUMA, stream=stream)]
        ctxs = systems
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sweeps = args.sweeps
    step_attempts = len(systems) * P * sweeps * N
    launches_per_step = len(systems) * 5  # sweep, counter advance, merge, recursion, thresholds

    def step(kevents=None):
        sharded_step(systems, sweeps, kevents, stream)

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            step()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    kev = []
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        t0.record(stream)
        for _ in range(args.steps):
            flush.zero_()  # L2 flush between timed steps (written on the same stream)
            step(kev)
        t1.record(stream)
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = t0.elapsed_time(t1)
    ms_t = torch.tensor([ms], device="cuda")
    if world > 1:
        torch.distributed.all_reduce(ms_t, op=torch.distributed.ReduceOp.MAX)
        torch.distributed.barrier()
    ms = float(ms_t.item())
    value = world * step_attempts * args.steps / (ms / 1e3)
    sweep_ms = statistics.mean(a.elapsed_time(b) for a, b in kev)

    # end to end through the C ABI: state in from pinned host memory, state out, every step
    bufs = []
    for s in ctxs:
        n = m.muca_get_state(s.h, None)
        t = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        buf = t.numpy()
        m.muca_get_state(s.h, buf)
        bufs.append((t, buf))
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    h0 = time.perf_counter()
    for _ in range(e2e_steps):
        for s, c, (_, buf) in zip(systems, ctxs, bufs):
            m.muca_set_state(c.h, buf)
            s.iterate(sweeps)
            s.merge_and_update()
            m.muca_get_state(c.h, buf)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - h0
    state_bytes = sum(b.nbytes for _, b in bufs)
    e2e = {"value": world * step_attempts * e2e_steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
           "d2h_bytes_per_step": state_bytes, "steps": e2e_steps}
    if world > 1:
        v = torch.tensor([e2e_s], device="cuda")
        torch.distributed.all_reduce(v, op=torch.distributed.ReduceOp.MAX)
        e2e["value"] = world * step_attempts * e2e_steps / float(v.item())

    if rank != 0:
        torch.distributed.destroy_process_group()
        return
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    f_mhz = ck["sm_mhz"] if ck else 2070.0
    peak_tinst = sms * 4 * 32 * f_mhz * 1e6 / 1e12
    achieved_tinst = P * sweeps * N * INSTR_PER_ATTEMPT / (sweep_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved_tinst, "peak": peak_tinst, "unit": "Tinst/s",
                "frac": achieved_tinst / peak_tinst, "traffic": TRAFFIC_PER_LAUNCH,
                "kernel": "k_sweep_spin_tn (code form; Ising L=32 MUCA and MUMA)", "kernel_ms": sweep_ms,
                "peak_basis": "%d SMs x 4 schedulers x 32 lanes x %.0f MHz (median sampled SM clock)" % (sms, f_mhz),
                "instr_per_attempt": INSTR_PER_ATTEMPT}
    chain_rate = P * f_mhz * 1e6 / CHAIN_CYCLES
    kernel_rate = P * sweeps * N / (sweep_ms / 1e3)
    roofline["chain_bound"] = {"cycles_per_attempt": CHAIN_CYCLES, "attempts_per_s": chain_rate,
                               "achieved_attempts_per_s": kernel_rate, "frac": kernel_rate / chain_rate,
                               "basis": "p x f_SM / cycles of one walker's chain with its scheduler to itself"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": "ising2d_L32_p8192_muca+muma", "L": L, "p": P, "systems": 2,
                       "sweeps_per_step": sweeps, "beta_muma": BETA_MUMA,
                       "l2": "flushed between steps (256 MiB write on the stream)",
                       "parallelism": "walkers (one chain per thread)" if world == 1 else
                       ("walkers of each system sharded over %d GPUs (%d a GPU), one histogram all-reduce "
                        "per system per iteration" % (world, P) if sharded else "independent replicas, one per GPU")},
            "e2e": e2e, "gpu_launches": launches_per_step * args.steps, "roofline": roofline,
            "clocks": ck}
    if not args.no_extras:
        line["batched_mix"] = run_mix(m, torch)
        line["potts_q8_L32"] = run_potts(m, torch)
        line["potts_q10_L64"] = run_potts64(m, torch)
        line["polymer"] = run_polymer(m, torch)
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_sample(args.cpu_sweeps, 5)
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "all":
        import torch

        import paper_1312_2213_gb300 as m

        m.load()
        res = {"mix": run_mix, "polymer": run_polymer, "potts": run_potts,
               "potts64": run_potts64}[args.workload](m, torch)
        print(json.dumps({"workload": args.workload, **res}), flush=True)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
