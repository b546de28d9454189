"""Sharded runs on the GPU: two gloo ranks (spawned processes, both on this GPU; no kernel waits
on another rank, the exchange is a host all-reduce) each run half of the walkers through the C ABI
(muca_merge_open + all-reduce + muca_update_with).  Weights, histograms and lattices must equal one
context of all walkers bit for bit."""
import json
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
CASES = [(m.ISING2D, 16, 2, 64, 7, 4, 20), (m.POTTS2D, 16, 8, 70, 9, 3, 15)]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


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
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1312_2213_gb300.shard import ShardedMuca

    system, L, q, p, seed, iters, sweeps = case
    s = ShardedMuca(system, L, q, p, seed)
    for _ in range(iters):
        s.iterate(sweeps)
        s.merge_and_update()
    np.save(os.path.join(out_dir, "lnW_%d.npy" % rank), s.ctx.lnW())
    np.save(os.path.join(out_dir, "H_%d.npy" % rank), s.ctx.histogram())
    np.save(os.path.join(out_dir, "spins_%d.npy" % rank), s.ctx.spins())
    met = s.metrics()  # summed over the ranks
    with open(os.path.join(out_dir, "metrics_%d.json" % rank), "w") as f:
        json.dump(met, f)
    dist.barrier()
    s.close()
    dist.destroy_process_group()


@pytest.mark.parametrize("case", CASES)
def test_two_shards_equal_one_context(tmp_path, case):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path), case), nprocs=world, join=True,
                       start_method="spawn")
    system, L, q, p, seed, iters, sweeps = case
    g = m.Muca(system, L, q, p, seed)
    for _ in range(iters):
        g.iterate(sweeps)
        g.merge_and_update()
    for rank in range(world):
        np.testing.assert_array_equal(np.load(tmp_path / ("lnW_%d.npy" % rank)).view(np.uint64),
                                      g.lnW().view(np.uint64))
        np.testing.assert_array_equal(np.load(tmp_path / ("H_%d.npy" % rank)), g.histogram())
    spins = np.concatenate([np.load(tmp_path / ("spins_%d.npy" % r)) for r in range(world)])
    np.testing.assert_array_equal(spins, g.spins())
    gm = g.metrics()
    for rank in range(world):
        with open(tmp_path / ("metrics_%d.json" % rank)) as f:
            sm = json.load(f)
        for k in ("accepted", "tunnelling_events", "accepted_total", "tunnelling_events_total", "sweeps",
                  "iteration", "acceptance_rate"):
            assert sm[k] == gm[k], k
