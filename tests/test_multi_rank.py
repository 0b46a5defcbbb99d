"""The multi-rank host logic of the benchmark, run as two gloo ranks on CPU.

The annealer does not shard (one graph per GPU; more GPUs run more replicas),
so the only cross-rank steps are the replica seed offset, the max-over-ranks
time and the whole-job throughput. These run here exactly as under torchrun,
with the gloo backend in place of NCCL.
"""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        assert (w, r, local) == (world, rank, rank)
        local_ms = 100.0 + 50.0 * rank           # rank 1 is the slow one
        t = bench.max_over_ranks(local_ms, world, dist, "cpu")
        seed = bench.replica_seed(1, rank)
        seeds = [None] * world
        dist.all_gather_object(seeds, seed)
        value = bench.job_throughput(1000.0, world, t / 1e3)
        out.put((rank, t, seeds, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_max_time_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort()
    for rank, t, seeds, value in res:
        assert t == 150.0                        # slowest rank's time on every rank
        assert len(set(seeds)) == 2              # distinct replicas
        assert value == pytest.approx(2 * 1000.0 / 0.150)


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, None, "cpu") == 3.5
    assert bench.replica_seed(7, 0) == 7
    assert bench.job_throughput(10.0, 1, 2.0) == 5.0
