"""The sharded form of the parallel scheme (Fig. 1 with walkers split over processes, one per
GPU): each rank runs the walkers of its contiguous id range, the open histograms are summed with
an all-reduce, and every rank runs the identical recursion.  Checked here with world_size-2 gloo
ranks on the CPU (using the oracle for the walkers): the merged histogram, ln W and the walkers'
lattices equal those of one process that runs all walkers."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

SYSTEM, L, Q, P, SEED, ITERS, SWEEPS = 1, 8, 5, 24, 31, 3, 60


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle

    r = oracle.Run(SYSTEM, L, Q, P, SEED)
    r.init()
    w0, w1 = rank * P // world, (rank + 1) * P // world
    for _ in range(ITERS):
        r.iterate_range(SWEEPS, w0, w1, 2)
        r.advance(SWEEPS)
        h = torch.from_numpy(r.open_histogram().astype(np.int64))
        dist.all_reduce(h, op=dist.ReduceOp.SUM)          # the one exchange per iteration
        r.set_open_histogram(h.numpy().astype(np.uint64))
        r.update()
    np.save(os.path.join(out_dir, "lnW_%d.npy" % rank), r.lnW())
    np.save(os.path.join(out_dir, "H_%d.npy" % rank), r.histogram())
    np.save(os.path.join(out_dir, "spins_%d.npy" % rank), r.spins()[w0:w1])
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_one_process(tmp_path, orc):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    ref = orc.Run(SYSTEM, L, Q, P, SEED)
    ref.init()
    for _ in range(ITERS):
        ref.iterate(SWEEPS, 4)
        ref.update()
    for rank in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / ("lnW_%d.npy" % rank)).view(np.uint64),
                                      ref.lnW().view(np.uint64))
        np.testing.assert_array_equal(np.load(tmp_path / ("H_%d.npy" % rank)), ref.histogram())
    spins = np.concatenate([np.load(tmp_path / ("spins_%d.npy" % r)) for r in range(world)])
    np.testing.assert_array_equal(spins, ref.spins())


def _failing_rank_main(rank, world, port, out_dir):
    """Rank 1 leaves after the first iteration (between iterations, nothing in flight); rank 0
    sees the next all-reduce fail, continues alone in a new single-rank group and merges only its
    own walkers from then on."""
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import datetime

    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=20))
    import oracle

    r = oracle.Run(SYSTEM, L, Q, P, SEED)
    r.init()
    w0, w1 = rank * P // world, (rank + 1) * P // world
    group_alive = True
    for it in range(ITERS + 1):
        if rank == 1 and it == 1:
            os._exit(0)  # the failure: this rank is gone
        r.iterate_range(SWEEPS, w0, w1, 2)
        r.advance(SWEEPS)
        h = torch.from_numpy(r.open_histogram().astype(np.int64))
        if group_alive:
            try:
                dist.all_reduce(h, op=dist.ReduceOp.SUM)
            except Exception:
                # survivors regroup (here: rank 0 alone) and merge their own walkers only
                group_alive = False
                with open(os.path.join(out_dir, "failed_at.txt"), "w") as f:
                    f.write(str(it))
        r.set_open_histogram(h.numpy().astype(np.uint64))
        r.update()
    np.save(os.path.join(out_dir, "lnW_survivor.npy"), r.lnW())
    np.save(os.path.join(out_dir, "H_survivor.npy"), r.histogram())


def test_survivor_continues_after_a_rank_fails(tmp_path, orc):
    world = 2
    ctx = mp.start_processes(_failing_rank_main, args=(world, _free_port(), str(tmp_path)),
                             nprocs=world, join=False, start_method="spawn")
    while not ctx.join(timeout=120):
        pass
    failed_at = int((tmp_path / "failed_at.txt").read_text())
    assert failed_at == 1
    ref = orc.Run(SYSTEM, L, Q, P, SEED)
    ref.init()
    for it in range(ITERS + 1):
        if it < failed_at:
            ref.iterate(SWEEPS, 4)             # both ranks' walkers merged
        else:
            ref.iterate_range(SWEEPS, 0, P // world, 2)   # the survivor's walkers only
            ref.advance(SWEEPS)
        ref.update()
    np.testing.assert_array_equal(np.load(tmp_path / "lnW_survivor.npy").view(np.uint64), ref.lnW().view(np.uint64))
    np.testing.assert_array_equal(np.load(tmp_path / "H_survivor.npy"), ref.histogram())
