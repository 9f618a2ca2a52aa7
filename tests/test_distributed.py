"""Multi-rank paths on CPU through torch.distributed.run (127.0.0.1, gloo): the benchmark's rank
plumbing (barrier, max over ranks of the step time), and the sharded update (receiver-sharded
Green solves, one exchange to frequency shards, the penalty from one all-reduce, the multipliers
summed over ranks) with oracle-backed contexts against the unsharded pipeline."""
import json
import os
import re
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_gloo_ranks_barrier_and_max():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "dist_helper.py")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=240, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    # the ranks' lines may interleave on the shared stdout
    rows = [json.loads(m) for m in re.findall(r"\{[^{}]*\}", r.stdout)]
    assert sorted(x["rank"] for x in rows) == [0, 1]
    assert all(x["ws"] == 2 for x in rows)
    assert all(x["max"] == 1.5 for x in rows)


@pytest.mark.parametrize("ws", [2, 3])
def test_sharded_update_equals_unsharded(ws):
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes", "1", "--nproc-per-node", str(ws),
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "tests", "dist_sharded_helper.py")]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, env=env, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-3000:]
    rows = [json.loads(m) for m in re.findall(r"\{.*\}", r.stdout)]
    assert len(rows) == 1 and rows[0]["ws"] == ws
    x = rows[0]
    # 7 receivers and 5 frequencies in contiguous blocks over the ranks
    assert [b[1] - b[0] for b in x["blocks"]] == [7 // ws + (i < 7 % ws) for i in range(ws)]
    assert [b[1] - b[0] for b in x["fblocks"]] == [5 // ws + (i < 5 % ws) for i in range(ws)]
    # per-frequency work is the same computation; only the order of the diagonal sum and of the
    # sum over frequencies in the synthesis differ
    assert x["mu_rel"] <= 1e-14
    assert x["q_max_abs"] <= 1e-12
    assert x["mult_rel"] <= 1e-12
