"""The sharded exchange over NCCL, as bench.py --gpus N runs it: two ranks, one GPU each
(torch.distributed with the nccl backend, NVLS off), each holding half of the walkers of one
system; after every iteration's sweeps the ranks all-reduce their open histograms on the device
(muca_merge_open + NCCL all_reduce + muca_update_with).  Weights, histograms and lattices must equal
one context of all walkers bit for bit.  Needs two GPUs: skipped where fewer are visible."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import paper_1312_2213_gb300 as m  # noqa: E402

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CASES = [(m.ISING2D_MUMA, 32, 2, 256, 7, 3, 20), (m.POTTS2D, 16, 8, 130, 9, 3, 15)]


@pytest.fixture(scope="module", autouse=True)
def _two_gpus():
    if not torch.cuda.is_available() or torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir, case):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    os.environ["NCCL_NVLS_ENABLE"] = "0"
    torch.cuda.set_device(rank)
    dist.init_process_group("nccl", rank=rank, world_size=world)
    from paper_1312_2213_gb300.shard import ShardedMuca

    system, L, q, p, seed, iters, sweeps = case
    s = ShardedMuca(system, L, q, p, seed, beta=0.4407 if system == m.ISING2D_MUMA else None)
    for _ in range(iters):
        s.iterate(sweeps)
        s.merge_and_update()
    np.save(os.path.join(out_dir, "lnW_%d.npy" % rank), s.ctx.lnW())
    np.save(os.path.join(out_dir, "H_%d.npy" % rank), s.ctx.histogram())
    np.save(os.path.join(out_dir, "spins_%d.npy" % rank), s.ctx.spins())
    dist.barrier()
    s.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", CASES)
def test_two_nccl_ranks_equal_one_context(tmp_path, case):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), case), nprocs=world, join=True,
                       start_method="spawn")
    system, L, q, p, seed, iters, sweeps = case
    g = m.Muca(system, L, q, p, seed, beta=0.4407 if system == m.ISING2D_MUMA else None)
    for _ in range(iters):
        g.iterate(sweeps)
        g.merge_and_update()
    for rank in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / ("lnW_%d.npy" % rank)).view(np.uint64),
                                      g.lnW().view(np.uint64))
        np.testing.assert_array_equal(np.load(tmp_path / ("H_%d.npy" % rank)), g.histogram())
    spins = np.concatenate([np.load(tmp_path / ("spins_%d.npy" % r)) for r in range(world)])
    np.testing.assert_array_equal(spins, g.spins())
