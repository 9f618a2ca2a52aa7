"""Run by tests/test_distributed.py under torch.distributed.run (one process per rank): the
benchmark's rank plumbing (process group, barrier, max over ranks) on the gloo backend."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

ws, rank, local = bench._dist()
t = bench._max_over_ranks(ws, 0.5 + rank)  # per-rank "time"; the slowest rank sets the step time
bench._barrier(ws)
print(json.dumps({"rank": rank, "local": local, "ws": ws, "max": t}), flush=True)
