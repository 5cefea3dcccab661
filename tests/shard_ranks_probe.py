"""Helper of tests/test_sharding_cpu.py, run under torch.distributed.run by
bench.relaunch: each rank builds its shard of the weak-scaling grid with
bench.shard_rect and reports the global rows it holds; rank 0 prints one JSON
line with the world size and every rank's rows. gloo, no GPU."""
import argparse
import json
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import bench  # noqa: E402
from test_sharding_cpu import global_rows  # noqa: E402


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--side", type=int, default=16)
    args = ap.parse_args()
    ws, rank, _ = bench.dist_setup()
    dist.init_process_group("gloo")
    rows = torch.tensor(global_rows(bench.shard_rect(rank, ws, args.side), ws, args.side),
                        dtype=torch.int64)
    allrows = [torch.zeros(args.side, dtype=torch.int64) for _ in range(ws)]
    dist.all_gather(allrows, rows)
    if rank == 0:
        print(json.dumps({"n_gpus": ws, "rows": [r.tolist() for r in allrows]}), flush=True)
    dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
