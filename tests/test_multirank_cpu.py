"""The multi-GPU path on CPU: world_size 2 over gloo (127.0.0.1).

Chains are independent, so the path shards by chains with no collective on
the data path.  Two ranks each run the FP64 oracle on their shard (chain
offset rank x C, same seed) and the gathered chains equal one run of all the
chains; the bench's per-rank seeds are distinct and its job throughput uses
the slowest rank's time (max over ranks through the process group).
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402
import oracle  # noqa: E402
import workloads  # noqa: E402

C = 6       # chains per rank
STEPS = 5


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = workloads.small(n_chains=C * world)
        shard = inst.X0[rank * C:(rank + 1) * C]
        X, _, _ = oracle.run(inst.A, inst.b, shard, STEPS, seed=11, chain_offset=rank * C,
                             n_threads=1)
        gathered = [torch.zeros((C, inst.d), dtype=torch.float64) for _ in range(world)]
        dist.all_gather(gathered, torch.from_numpy(X))
        # the bench's aggregation: each rank reports its own time, the job
        # takes the slowest
        ms = 10.0 + rank
        ms_max = bench.max_over_ranks(world, ms)
        value = bench.job_throughput(world, C, STEPS, ms_max)
        seeds = [torch.zeros(1, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(seeds, torch.tensor([bench.rank_seed(11, rank)], dtype=torch.int64))
        if rank == 0:
            out["X"] = torch.cat(gathered).numpy()
            out["ms_max"] = ms_max
            out["value"] = value
            out["seeds"] = [int(t.item()) for t in seeds]
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_chains_and_aggregate():
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    inst = workloads.small(n_chains=C * world)
    want, _, _ = oracle.run(inst.A, inst.b, inst.X0, STEPS, seed=11, n_threads=1)
    np.testing.assert_array_equal(res["X"], want)
    assert res["ms_max"] == 11.0
    assert res["value"] == pytest.approx(world * C * STEPS / 0.011)
    assert len(set(res["seeds"])) == world
