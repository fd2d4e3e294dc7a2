"""Host logic of the N-process benchmark on CPU: two gloo ranks plan disjoint
seed ranges and agree on the max-over-ranks timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, _ = bench.dist_env()
    seeds = [bench.rank_seed_base(r) + s for s in range(10)]
    slowest = bench.max_over_ranks(1.0 + r, w, "cpu")
    dist.barrier()
    out.put((r, w, seeds, slowest))
    dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_seeds_and_max_timing():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[0] for r in res] == [0, 1] and all(r[1] == 2 for r in res)
    assert not set(res[0][2]) & set(res[1][2])          # independent problems per rank
    assert all(r[3] == 2.0 for r in res)                # every rank sees the slowest time


def test_single_rank_is_identity():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5
