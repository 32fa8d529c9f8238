"""The multi-rank logic of the benchmark on two gloo ranks (CPU): disjoint pairs per rank,
the timed region's end taken as the slowest rank's, whole-job throughput over all ranks."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seeds = bench.pair_seeds(rank, 4)
        ms = bench.max_over_ranks(100.0 + 50.0 * rank, world)   # rank 1 is the slow one
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        out.put((rank, ms, gathered, bench.weak_value(10, 4, world, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_disjoint_pairs_and_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, gathered, value in res:
        assert ms == 150.0                                    # max over ranks
        assert not set(gathered[0]) & set(gathered[1])        # no pair is shared
        assert value == pytest.approx(10 * 4 * 2 / 0.150)     # all ranks' pairs / slowest time
