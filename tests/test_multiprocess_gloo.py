"""Multi-process (one process per GPU) host logic, run as two gloo ranks on the CPU: the frame
sharding is a deterministic partition every rank computes alike, and the benchmark's barrier and
max-over-ranks step-time reduction behave as its JSON contract needs. No GPU is used."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1910_11872_gb300 import shard

SHAPES = [(1024, 1024), (256, 512), (2048, 1024), (512, 512), (768, 256), (1024, 512), (256, 256)]


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench  # the benchmark's own multi-rank helpers

    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    mine = shard.my_frames(SHAPES, rank, world)
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    bench.barrier(world)
    step_ms = 10.0 * (rank + 1)
    mx = bench.max_over_ranks(world, step_ms)
    q.put((rank, gathered, mx))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, mx in results:
        assert mx == 20.0  # the slowest rank sets the step time
        flat = sorted(i for part in gathered for i in part)
        assert flat == list(range(len(SHAPES)))  # every frame exactly once
        assert gathered == shard.shard_frames(SHAPES, world)  # all ranks agree


@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_shard_balance(world):
    parts = shard.shard_frames(SHAPES, world)
    loads = [sum(SHAPES[i][0] * SHAPES[i][1] for i in p) for p in parts]
    assert sorted(i for p in parts for i in p) == list(range(len(SHAPES)))
    biggest = max(h * w for h, w in SHAPES)
    assert max(loads) - min(loads) <= biggest
