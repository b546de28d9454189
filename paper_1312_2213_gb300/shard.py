"""One system whose walkers are split over processes, typically one per GPU: the paper's Fig. 1
scheme with the per-iteration exchange as a single all-reduce of the histogram.

Rank r of a group of size n runs walkers [r p / n, (r+1) p / n) of the system as a context with
`walker_offset` set to its first walker, so its random streams are exactly those the walkers
have in one context of all p.  After the sweeps each rank sums its open histogram into a device
buffer (`muca_merge_open`), the buffers are added with `torch.distributed.all_reduce` (NCCL on
the device buffer; other backends through a host copy), and every rank closes the iteration with
the summed histogram (`muca_update_with`).  The ranks then hold identical weights, and together
equal one context of all walkers bit for bit.

A rank that fails is seen by the others as a failing collective.  The survivors can carry on in
a new group (`set_group`): their walkers keep their state, and from then on the merge runs over
the surviving walkers only.
"""
from __future__ import annotations

import torch
import torch.distributed as dist

from . import Muca


def shard_range(p: int, rank: int, world: int) -> tuple[int, int]:
    """Contiguous walker range [w0, w1) of a rank."""
    return rank * p // world, (rank + 1) * p // world


class ShardedMuca:
    """One rank's shard of a system.  `ctx_factory` builds the rank's context (default: a Muca
    context on the current CUDA device); anything with the same iterate / merge_open / update_with
    / metrics methods works, which lets the exchange itself be tested without a GPU."""

    def __init__(self, system: int, L: int, q: int, p: int, seed: int, group=None, ctx_factory=None,
                 device: str = "cuda", **kw):
        self.group = group
        rank, world = dist.get_rank(group), dist.get_world_size(group)
        self.w0, self.w1 = shard_range(p, rank, world)
        if self.w1 <= self.w0:
            raise ValueError("more ranks than walkers")
        self.ctx = (ctx_factory or Muca)(system, L, q, self.w1 - self.w0, seed, walker_offset=self.w0, **kw)
        self.B = self.ctx.B
        self.device = device
        self.buf = torch.zeros(self.B, dtype=torch.int64, device=device)

    def set_group(self, group):
        """Continue in another process group (e.g. the survivors after a rank failed)."""
        self.group = group

    def iterate(self, sweeps: int):
        self.ctx.iterate(sweeps)

    def merge_and_update(self, want_flat: bool = False):
        """Sum the open histograms of all ranks and close the iteration on this rank."""
        self.ctx.merge_open(self.buf)
        if dist.get_backend(self.group) == "nccl" or self.buf.device.type == "cpu":
            dist.all_reduce(self.buf, group=self.group)
        else:
            host = self.buf.cpu()
            dist.all_reduce(host, group=self.group)
            self.buf.copy_(host)
        if self.buf.device.type == "cuda":
            torch.cuda.synchronize()
        return self.ctx.update_with(self.buf, want_flat)

    def metrics(self) -> dict:
        """The last closed iteration's metrics summed over the ranks of the group (each rank
        counts its own walkers); the acceptance rate is over all walkers."""
        d = self.ctx.metrics()
        keys = ("accepted", "tunnelling_events", "accepted_total", "tunnelling_events_total")
        t = torch.tensor([d[k] for k in keys] + [self.w1 - self.w0], dtype=torch.int64)
        if dist.get_backend(self.group) == "nccl":
            t = t.to(self.device)
        dist.all_reduce(t, group=self.group)
        t = t.cpu()
        out = dict(d)
        out.update({k: int(v) for k, v in zip(keys, t[:4])})
        p = int(t[4])
        attempts = p * self.ctx.N * d["sweeps"]
        out["acceptance_rate"] = out["accepted"] / attempts if attempts else float("nan")
        return out

    def close(self):
        self.ctx.close()
