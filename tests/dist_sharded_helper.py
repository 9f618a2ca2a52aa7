"""Run by tests/test_distributed.py under torch.distributed.run (one gloo process per rank): the
sharded update (paper_2512_16642_gb300.sharded) with oracle-backed contexts against the unsharded
oracle pipeline on the same tiny case; rank 0 prints the largest differences."""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

import numpy as np  # noqa: E402
import torch  # noqa: E402
import torch.distributed as dist  # noqa: E402

import synth  # noqa: E402
from paper_2512_16642_gb300 import sharded  # noqa: E402
from sharded_oracle_ctx import OracleContext  # noqa: E402

dist.init_process_group("gloo")
rank, ws = dist.get_rank(), dist.get_world_size()
c = synth.case_tiny(seed=21, nz=10, nx=14, nsponge=4, nrec=7, nt=60)
c["freqs"] = np.array([11.0, 17.0, 23.0, 29.0, 35.0])
geom = {k: c[k] for k in ("nz", "nx", "dz", "dx", "nsponge", "sponge_R", "dt", "nt", "rec_iz",
                          "rec_ix", "freqs")}
vel = torch.from_numpy(np.float32(c.vel_true).astype(np.float64))
resid = torch.from_numpy(np.random.default_rng(3).standard_normal((3, 7, 60)))
alpha = 1e-2

shard = sharded.Shard(geom, rank, ws, context_factory=OracleContext)
mult = torch.zeros((3, 7, 60), dtype=torch.float64)
mu = sharded.update(shard, vel, resid, mult, alpha)
k0, k1 = shard.kb[rank]
Q_local = shard.hess_ctx.Q if shard.hess_ctx is not None else np.zeros((0, 7, 7))

# the unsharded pipeline (all receivers, all frequencies) on every rank
ref = OracleContext(*(geom[k] for k in ("nz", "nx", "dz", "dx", "nsponge", "sponge_R", "dt", "nt",
                                        "rec_iz", "rec_ix", "freqs")))
ref.green(vel)
ref.hessian()
mu_ref = alpha * ref.diag_sum() / (c.freqs.size * 7)
ref.set_mu(mu_ref)
ref.factor()
m_ref = torch.zeros_like(mult)
ref.deblur(resid, m_ref)

dq = float(np.max(np.abs(Q_local - ref.Q[k0:k1]))) if k1 > k0 else 0.0
out = torch.tensor([abs(mu - mu_ref) / mu_ref, dq, float((mult - m_ref).abs().max() / m_ref.abs().max())],
                   dtype=torch.float64)
dist.all_reduce(out, op=dist.ReduceOp.MAX)
if rank == 0:
    print(json.dumps({"ws": ws, "mu_rel": out[0].item(), "q_max_abs": out[1].item(),
                      "mult_rel": out[2].item(), "blocks": shard.rb, "fblocks": shard.kb}), flush=True)
dist.destroy_process_group()
