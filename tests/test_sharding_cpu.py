"""Multi-GPU layout on the CPU: world-size-2 gloo ranks take the interleaved
rows i = r (mod N) of the (N*1024) x 1024 weak-scaling grid, which together
cover it once, and the timing is the max over ranks. `bench.py --gpus N`
starts N ranks under torch.distributed.run. No GPU and no data-path
collective."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def global_rows(rect, world, side):
    """Global row index of each row of a shard's cell-centred grid."""
    re0, re1 = bench.RECT[:2]
    dre = (re1 - re0) / (world * side)
    x = rect[0] + (np.arange(side) + 0.5) * (rect[1] - rect[0]) / side
    g = (x - re0) / dre - 0.5
    assert np.allclose(g, np.round(g), atol=1e-6)
    return np.round(g).astype(int)


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    rect = bench.shard_rect(rank, world, side=8)
    rows = torch.tensor(global_rows(rect, world, 8), dtype=torch.int64)
    allrows = [torch.zeros(8, dtype=torch.int64) for _ in range(world)]
    dist.all_gather(allrows, rows)
    t = torch.tensor([0.5 + rank], dtype=torch.float64)    # this rank's elapsed time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        out.put(([r.tolist() for r in allrows], float(t.item())))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_interleaved_shards_cover_the_grid_once(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    rows, tmax = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    covered = np.zeros(world * 8, dtype=int)
    for r, rr in enumerate(rows):
        assert all(g % world == r for g in rr)      # rank r holds rows r mod N
        covered[rr] += 1
    assert np.all(covered == 1)
    assert tmax == 0.5 + (world - 1)


def test_one_rank_is_the_whole_grid():
    rect = bench.shard_rect(0, 1)
    assert rect == bench.RECT


@pytest.mark.parametrize("world", [2, 4, 8])
def test_every_shard_spans_the_same_range(world):
    """Each rank's rows spread over the whole real range (the same mix of
    cheap and expensive points), offset by one global row per rank."""
    re0, re1 = bench.RECT[:2]
    dre = (re1 - re0) / (world * bench.SIDE)
    for r in range(world):
        rows = global_rows(bench.shard_rect(r, world), world, bench.SIDE)
        assert rows[0] == r and rows[-1] == world * (bench.SIDE - 1) + r
        assert np.all(np.diff(rows) == world)
    a0 = bench.shard_rect(0, world)[0]
    a1 = bench.shard_rect(1, world)[0]
    assert abs((a1 - a0) - dre) < 1e-12


def test_gpus_flag_starts_one_process_per_rank():
    """The launcher bench.py uses for --gpus N (torch.distributed.run, N ranks
    on 127.0.0.1), driving a helper that builds each rank's shard with
    bench.shard_rect on gloo: rank 0 sees N ranks whose rows cover the grid
    once."""
    out = bench.relaunch(2, ["--side", "16"], script=os.path.join(HERE, "shard_ranks_probe.py"),
                         capture_output=True, text=True, timeout=300,
                         env=dict(os.environ, PYTHONPATH=os.pathsep.join(sys.path)))
    assert out.returncode == 0, out.stderr[-3000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["n_gpus"] == 2
    rows = sorted(g for rr in d["rows"] for g in rr)
    assert rows == list(range(2 * 16))
