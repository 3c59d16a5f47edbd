"""The N > 1 path of bench.py on CPU: two gloo ranks, each a replica of the
workload with its own seed, reduce their step times to the maximum (no data
exchange between replicas). No GPU involved."""

import os
import sys

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, times, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = bench.max_over_ranks(times[rank], world)
    seed = bench.replica_seed(rank)
    dist.barrier()
    q.put((rank, t, seed))
    dist.destroy_process_group()


@pytest.mark.parametrize("times", [(0.010, 0.025), (0.5, 0.2)])
def test_two_ranks_take_the_slowest(times):
    import random
    port = 29500 + random.randint(0, 2000)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, times, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert {r: t for r, t, _ in got} == {0: max(times), 1: max(times)}
    assert len({s for _, _, s in got}) == 2      # replicas use different inputs


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.123, 1) == 0.123
