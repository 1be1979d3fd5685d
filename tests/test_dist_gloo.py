"""The multi-GPU bench path is replicas only: each rank runs the whole workload and the job
rate is all ranks' work over the slowest rank's time.  Checked here with two CPU ranks over
the gloo backend (no GPU)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = 10.0 + 5.0 * rank                     # rank 1 is the slow replica
    slowest = bench.max_over_ranks(ms, dist, "cpu")
    rate = bench.whole_job_rate(world, 1000.0, slowest)
    out[rank] = (slowest, rate, bench.dist_env())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_aggregation_two_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        slowest, rate, env = res[rank]
        assert slowest == 15.0
        assert rate == pytest.approx(2 * 1000.0 / 0.015)
        assert env == (2, rank, 0)
