"""The benchmark's multi-GPU leg on the CPU: two gloo ranks build the workload exactly as
`bench.py --gpus 2` does (bench.make_sharded_systems: each system's walkers split over the
ranks, weak scaling) and run the bench's own step (bench.sharded_step: sweeps, then one
histogram all-reduce per system and the recursion), with oracle-backed contexts standing in for
the CUDA ones.  Every rank must end with the weights and histogram of one process that runs all
walkers of each system (Fig. 1: the merge is a plain sum, the recursion is the same on every rank)."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
P_PER_RANK, SWEEPS, STEPS = 8, 4, 2


class OracleShard:
    """A shard context backed by the oracle: walkers [w0, w0 + p) of a run of the same seed."""

    def __init__(self, system, L, q, p, seed, walker_offset=0, beta=None, stream=None):
        import oracle

        self.w0, self.w1 = walker_offset, walker_offset + p
        self.r = oracle.Run(system, L, q, self.w1, seed, beta=beta or 0.0)
        self.r.init()
        self.B = self.r.B

    def iterate(self, sweeps):
        self.r.iterate_range(sweeps, self.w0, self.w1, 2)
        self.r.advance(sweeps)

    def merge_open(self, buf):
        buf.copy_(torch.from_numpy(self.r.open_histogram().astype(np.int64)))

    def update_with(self, buf, want_flat=False):
        self.r.set_open_histogram(buf.numpy().astype(np.uint64))
        self.r.update()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    systems = bench.make_sharded_systems(None, rank, world, p_per_rank=P_PER_RANK, ctx_factory=OracleShard,
                                         device="cpu")
    assert [(s.w0, s.w1) for s in systems] == [(rank * P_PER_RANK, (rank + 1) * P_PER_RANK)] * 2
    for _ in range(STEPS):
        bench.sharded_step(systems, SWEEPS)
    for k, s in enumerate(systems):
        np.save(os.path.join(out_dir, "lnW_%d_%d.npy" % (k, rank)), s.ctx.r.lnW())
        np.save(os.path.join(out_dir, "H_%d_%d.npy" % (k, rank)), s.ctx.r.histogram())
    dist.barrier()
    dist.destroy_process_group()


def test_bench_sharded_leg_equals_one_process(tmp_path, orc):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    sys.path.insert(0, ROOT)
    import bench

    for k, (system, seed, beta) in enumerate(((0, 1, 0.0), (2, 1001, bench.BETA_MUMA))):
        ref = orc.Run(system, bench.L, 2, P_PER_RANK * world, seed, beta=beta)
        ref.init()
        for _ in range(STEPS):
            ref.iterate(SWEEPS, 4)
            ref.update()
        for rank in range(world):
            np.testing.assert_array_equal(np.load(tmp_path / ("lnW_%d_%d.npy" % (k, rank))).view(np.uint64),
                                          ref.lnW().view(np.uint64))
            np.testing.assert_array_equal(np.load(tmp_path / ("H_%d_%d.npy" % (k, rank))), ref.histogram())
