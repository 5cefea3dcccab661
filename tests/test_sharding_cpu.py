"""Multi-GPU layout on the CPU: world-size-2 gloo ranks take disjoint row
blocks of the (N*1024) x 1024 weak-scaling grid that together cover it once,
and the timing is the max over ranks. No GPU and no data-path collective."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rect, (r0, r1) = bench.shard_rows(rank, world, side=8)
    rows = torch.tensor([r0, r1], dtype=torch.int64)
    allrows = [torch.zeros(2, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allrows, rows)
    t = torch.tensor([0.5 + rank], dtype=torch.float64)    # this rank's elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put(([tuple(r.tolist()) for r in allrows], float(t.item()), rect))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_row_shards_cover_the_grid_once(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    rows, tmax, rect0 = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = np.zeros(world * 8, dtype=int)
    for r0, r1 in rows:
        covered[r0:r1] += 1
    assert np.all(covered == 1)
    assert tmax == 0.5 + (world - 1)
    # rank 0's block starts at the rectangle's left edge
    assert rect0[0] == bench.RECT[0]


def test_shard_rectangles_tile_the_real_range():
    world = 4
    edges = [bench.shard_rows(r, world)[0][:2] for r in range(world)]
    assert edges[0][0] == bench.RECT[0]
    assert abs(edges[-1][1] - bench.RECT[1]) < 1e-12
    for a, b in zip(edges, edges[1:]):
        assert abs(a[1] - b[0]) < 1e-12
