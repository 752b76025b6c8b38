"""Multi-rank host logic of the benchmark on CPU (gloo, world size 2).

The path shards by instance: every rank solves its own batch (weak scaling) or
its share of one batch under the work-weighted partition (strong scaling), and
the only cross-rank steps are a barrier and the maximum of the timed
durations.  These tests run that host logic on two gloo ranks without a GPU.
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


def _partition_worker(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2602_23967_b300 import partition as PT
    from paper_2602_23967_b300 import workloads as W

    # every rank computes its share of one fixed batch on its own (no list is
    # exchanged in the bench); here the shares are gathered only to check them
    qps = W.mpc_batch(count=96, seed=0)
    w = [PT.work_estimate(q, diagonal_q=True) for q in qps]
    mine = PT.partition(w, world)[rank]
    shares = [None] * world
    dist.all_gather_object(shares, mine)
    mine_bench = bench.instances(96, rank, world, "strong")
    sizes = [None] * world
    dist.all_gather_object(sizes, len(mine_bench))
    np.save(os.path.join(out_dir, f"part{rank}.npy"),
            np.array([len(set(sum(shares, []))), sum(len(s) for s in shares), max(PT.loads(w, shares)),
                      min(PT.loads(w, shares)), max(w), sum(sizes), len(mine_bench) == len(mine)],
                     dtype=np.float64))
    dist.destroy_process_group()


@pytest.mark.timeout(300)
def test_two_gloo_ranks_partition_one_batch_by_work(tmp_path):
    world = 2
    mp.start_processes(_partition_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       start_method="spawn", join=True)
    for r in range(world):
        distinct, total, hi, lo, wmax, bench_total, same_len = np.load(tmp_path / f"part{r}.npy")
        assert distinct == total == 96           # complete and disjoint
        assert hi - lo <= wmax                   # LPT balance: within one instance's work
        assert bench_total == 96 and same_len    # the bench's strong-scaling shares are these


def test_partition_properties():
    from paper_2602_23967_b300 import partition as PT
    rng = np.random.default_rng(0)
    for world in (1, 2, 3, 8):
        w = [int(v) for v in rng.integers(1, 1000, size=257)]
        parts = PT.partition(w, world)
        flat = sorted(sum(parts, []))
        assert flat == list(range(len(w)))
        ld = PT.loads(w, parts)
        assert max(ld) - min(ld) <= max(w)
        assert PT.partition(w, world) == parts          # deterministic
    # more ranks than instances: the extra ranks get nothing
    assert PT.partition([5, 3], 4) == [[0], [1], [], []]
    with pytest.raises(ValueError):
        PT.partition([1], 0)
