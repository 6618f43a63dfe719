"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs its own reconstruction (replicas, no data-path collective); the job time
is the maximum over ranks and the throughput counts all ranks' units."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    r, w, local = bench.dist_env()
    ms = 100.0 + 50.0 * rank                      # rank 1 is the slow one
    dist.barrier()
    slowest = bench.max_over_ranks(ms)
    rate = bench.aggregate_rate(1000, w, slowest)
    out.put((r, w, local, slowest, rate))
    dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate_gloo():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, (r, w, local, slowest, rate) in enumerate(results):
        assert (r, w, local) == (rank, world, rank)
        assert slowest == pytest.approx(150.0)
        assert rate == pytest.approx(1000 * 2 / 0.150)


def test_single_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(42.0) == 42.0
    assert bench.aggregate_rate(10, 1, 1000.0) == pytest.approx(10.0)
