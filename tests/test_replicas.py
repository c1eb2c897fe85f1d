"""The multi-GPU path is replicas only: every rank decodes its own shots, no data crosses ranks.

Runs bench.py's sharding and max-over-ranks timing helpers on two gloo ranks on the CPU.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, batch, out):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    from paper_2508_07879_gb300 import workloads as w
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        first, count = bench.shard(rank, world, batch)
        b = w.x_error_batch(w.hgp_code(400), 0.05, count, seed=2001, first_shot=first)
        slowest = bench.reduce_max(10.0 * (rank + 1))
        shards = [None] * world
        dist.all_gather_object(shards, (first, count))
        out.put((rank, slowest, shards, b.syndromes))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_replica_shards_and_job_time(world):
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    batch = 48
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, batch, out)) for r in range(world)]
    for p in procs:
        p.start()
    results = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    results.sort(key=lambda r: r[0])
    # every rank sees the slowest rank's time
    assert all(r[1] == 10.0 * world for r in results)
    # shards are disjoint, contiguous and cover [0, world*batch)
    shards = results[0][2]
    assert sorted(shards) == [(r * batch, batch) for r in range(world)]
    # the union of the shards' inputs is the single-process sequence
    import sys
    sys.path.insert(0, ROOT)
    from paper_2508_07879_gb300 import workloads as w
    whole = w.x_error_batch(w.hgp_code(400), 0.05, world * batch, seed=2001)
    np.testing.assert_array_equal(np.concatenate([r[3] for r in results]), whole.syndromes)


def test_reduce_max_without_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5) == 3.5
    assert bench.shard(3, 4, 100) == (300, 100)
