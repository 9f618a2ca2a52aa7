"""Multi-rank path of bench.py on CPU: two gloo ranks through torch.distributed.run (127.0.0.1).
Each rank of the benchmark runs one independent update (weak scaling, no data-path collective);
the only cross-rank steps are the barrier and the max over ranks of the step time, checked here."""
import json
import os
import re
import socket
import subprocess
import sys

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
