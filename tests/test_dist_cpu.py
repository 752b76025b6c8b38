"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards by instance: every rank solves its own batch and the only
cross-rank steps are a barrier and the maximum of the timed durations.  These
tests run that host logic on two gloo ranks without a GPU.
"""
import hashlib
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _digest(qps):
    h = hashlib.sha256()
    for q in qps:
        h.update(q.A.data.tobytes())
        h.update(q.lc.tobytes())
    return h.hexdigest()


def _worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    r, w, _ = bench.dist_env()
    assert (r, w) == (rank, world)
    qps = bench.instances(3, r)
    digests = [None] * world
    dist.all_gather_object(digests, _digest(qps))
    # each rank's local duration differs; the job's time is the slowest rank's
    local_ms = 100.0 + 50.0 * rank
    total = bench.max_over_ranks(local_ms, world)
    value = bench.job_throughput(world, 3, 2, total)
    dist.barrier()
    np.save(os.path.join(out_dir, f"rank{rank}.npy"),
            np.array([total, value, len(set(digests)), len(qps)], dtype=np.float64))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_shard_instances_and_take_max(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    rows = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    for total, value, distinct, count in rows:
        assert total == 150.0                        # max over ranks, seen by every rank
        assert value == pytest.approx(2 * 3 * 2 / 0.150)
        assert distinct == world                     # ranks solve different instances
        assert count == 3


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(1, 4096, 5, 1000.0) == pytest.approx(4096 * 5)
