#!/usr/bin/env python
"""Benchmark of the data-space Hessian hot path on the layered 921x301 workload.

One step = one model update through the whole path on one GPU: Green functions by finite
differences with the on-the-fly transform (231 receivers, 4000 steps, 26 frequencies 3-8 Hz),
Gram Hessians + mu, Cholesky factors, and the deblur of all 115 sources' residual gathers.

Prints one JSON line.  `value` is the Hessian build+factor time per update (s, lower is better),
timed with CUDA events on the stream the library launches on; `deblur_sources_per_s` and the
per-stage times ride along.  Inputs are device-resident and larger than L2 (the transforms are
16 GB, the residuals 425 MB), so nothing is flushed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--no-cpu-baseline]

--impl reference times the FP64 CPU oracle on a bounded sample of the same workload (its
Green solves, Gram, factorisation and deblur), extrapolated to a full update.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Hessian build+factor s/update"
UNIT = "s/update"
FALLBACK_HBM_GBS = 6800.0

# DRAM traffic (read + write bytes) per launch of the FD step and of the transform from the
# committed ncu capture (profiles/), valid only for the kernel sources it was taken from (sha256
# of csrc/fd.cu); None until a capture exists.
KERNEL_TRAFFIC = {"fd_sha256": "8afae4dbb4943cb9c3c79b80b5e97a5bc7d87578b94ef69c01d0f0998c9a03a3",
                  "k_fd_step": 32.13e6,   # 1.64 MB read + 30.49 MB write per launch (18 rows per warp)
                  "k_dft_tc": 48.10e9,    # 45.78 GB read + 2.33 GB write per 2048-level launch
                  "gram_sha256": "f9de315c9b531216c4542c842f967a76ddf97ec6b8c30623a20ace1b44982cd4",
                  # per launch at 231 receivers x 26 frequencies, by grid-sum splits (read + write)
                  "k_gram_tc": {8: 32.98e9, 16: 24.54e9, 32: 18.09e9}}


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--resid", choices=["model", "noise"], default="model",
                   help="residual gathers from forward modelling in the true and start models, or "
                        "seeded band-limited noise of the same shape (skips the modelling launches)")
    p.add_argument("--slice", action="store_true",
                   help="profiling slice: one batch of 16 receivers, nt 1024, no e2e or CPU baseline")
    p.add_argument("--slice-receivers", type=int, default=16,
                   help="receivers of the profiling slice (231 gives the full-size Hessian)")
    p.add_argument("--slice-nt", type=int, default=1024, help="time steps of the profiling slice")
    p.add_argument("--no-serving", action="store_true", help="skip the serving-form measurement")
    p.add_argument("--no-batched", action="store_true",
                   help="skip the batched-form (salt, three patches) leg of the default run")
    p.add_argument("--workload", choices=["layered", "salt", "deblur"], default="layered",
                   help="layered (the benchmark workload), the batched salt-patch form, or the "
                        "deblur kernels alone at the layered shape (for profiling captures)")
    p.add_argument("--precision", choices=["mixed", "fp32"], default="mixed",
                   help="Hessian arithmetic: bf16x3 tensor-core Gram (mixed) or FP32 CUDA-core Gram")
    p.add_argument("--sharded", action="store_true",
                   help="run the sharded update (receiver-sharded Green solves, one exchange to "
                        "frequency shards); the default whenever more than one rank runs")
    p.add_argument("--fd-kernel", type=int, choices=[0, 1, 2], default=0,
                   help="FD solver: 0 library choice, 1 resident, 2 one kernel per step")
    p.add_argument("--dft-chunk", type=int, default=2048,
                   help="levels per transform chunk (0 = library default 512; 2048 quarters the "
                        "transform's accumulator traffic of 512 for a 91 GB snapshot ring: "
                        "measured 1.6 %% faster than 1024 on the layered update)")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def _bf16_peak():
    """(TFLOP/s, kind): the sustained cuBLAS bf16 figure (the Gram runs inside a long step)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["bf16_tflops_sustained"]), "measured (sustained)"
    except Exception:
        return 1700.0, "fallback (sustained)"


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            out = self.parse(f)
        os.unlink(self.path)
        return out

    @staticmethod
    def parse(lines):
        """Summary of `--format=csv,noheader,nounits` lines of FIELDS: median SM clock, maximum
        SM clock and the throttle reasons seen active in any sample (None without samples)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------------
# distributed plumbing (one process per GPU; each rank runs its own independent update)
# ---------------------------------------------------------------------------------------------
def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        backend = "nccl" if _cuda() else "gloo"
        dist.init_process_group(backend)
    return ws, rank, local


def _cuda():
    import torch

    return torch.cuda.is_available()


def _barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def _max_over_ranks(ws, x):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], device="cuda" if _cuda() else "cpu", dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# the oracle on a bounded sample (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------------------------
def oracle_sample(c, green_steps=200, gram_receivers=None, deblur_sources=4):
    """Times the FP64 oracle on parts of one update and extrapolates to the full update.

    Green: `cores` receivers propagated concurrently (one per thread) for `green_steps` of the
    nt steps with the 26-frequency transform, scaled by (Nr / cores) x (nt / green_steps).
    Gram: Hessian of those receivers' transforms, scaled by (Nr / cores)^2.  Cholesky: all 26
    frequencies of a 231 x 231 Hermitian positive-definite matrix, in full.  Deblur: a few
    sources at full length, scaled by Ns / sources."""
    import numpy as np

    import oracle

    cores = os.cpu_count() or 1
    w = max(1, min(cores, 16))
    nr, nf, nt = c.rec_ix.size, c.freqs.size, c.nt
    grid = oracle.Grid(np.float32(c.vel_start).astype(np.float64), c.dz, c.dx, c.nsponge, c.sponge_R)
    sel = np.linspace(0, nr - 1, w).round().astype(int)
    t0 = time.perf_counter()
    gh = oracle.green_dtft(grid, c.rec_iz[sel], c.rec_ix[sel], c.freqs, c.dt, green_steps, workers=w)
    t_green = (time.perf_counter() - t0) * (nr / w) * (nt / green_steps)
    t0 = time.perf_counter()
    oracle.hessian_gram(gh)
    t_gram = (time.perf_counter() - t0) * (nr / w) ** 2
    rng = np.random.default_rng(0)
    A = rng.standard_normal((nf, nr, 2 * nr)) + 1j * rng.standard_normal((nf, nr, 2 * nr))
    Q = A @ A.conj().transpose(0, 2, 1) + nr * np.eye(nr)
    t0 = time.perf_counter()
    L = oracle.cholesky(Q)
    t_chol = time.perf_counter() - t0
    ns = c.src_ix.size
    resid = rng.standard_normal((deblur_sources, nr, nt))
    t0 = time.perf_counter()
    oracle.deblur(L, resid, c.freqs, c.dt)
    t_deb = (time.perf_counter() - t0) * ns / deblur_sources
    sample = (f"Green: {w} receivers x {green_steps} of {nt} steps (26-frequency transform) scaled "
              f"x{nr / w:.1f} x{nt / green_steps:.1f}; Gram of those {w} scaled x{(nr / w) ** 2:.0f}; "
              f"Cholesky of all {nf} frequencies in full; deblur of {deblur_sources} of {ns} sources "
              f"scaled x{ns / deblur_sources:.1f}")
    return {"build_factor_s": t_green + t_gram + t_chol, "green_s": t_green, "gram_s": t_gram,
            "chol_s": t_chol, "deblur_s": t_deb, "sources_per_s": ns / t_deb, "cores": w,
            "sample": sample}


def serving_error(serving):
    """Relative L2 error of each kept serving request's multipliers against the FP64 oracle
    (Cholesky of the set's Hessians, transform, solve, synthesis): part of the cpu_baseline leg."""
    import numpy as np

    import oracle

    errs, L_cache = [], {}
    for smp in serving["_samples"]:
        Q, f, dt, nt_rec = serving["_sets"][smp["set"]]
        if smp["set"] not in L_cache:
            L_cache[smp["set"]] = oracle.cholesky(Q.astype(np.complex128))
        ref = oracle.deblur(L_cache[smp["set"]], smp["resid"].astype(np.float64), f, dt, nt_ref=nt_rec)[0]
        errs.append(float(np.linalg.norm(smp["mult"] - ref) / np.linalg.norm(ref)))
    return errs


def _workload(c, extra=None):
    if c.rec_ix.size == 231 and c.nt == 4000:
        name = ("layered-faulted 921x301 (padded 961x341), dx 10 m, 231 receivers, 115 sources, "
                "nt 4000 dt 1 ms, 26 frequencies 3.0:0.2:8.0 Hz, mu 1e-2 mean diag")
    else:
        name = (f"profiling slice of the layered-faulted 921x301 workload: {c.rec_ix.size} receivers, "
                f"{c.src_ix.size} sources, nt {c.nt}")
    cfg = {"workload": name,
           "nz": c.nz, "nx": c.nx, "nsponge": c.nsponge, "nrec": int(c.rec_ix.size),
           "nsrc": int(c.src_ix.size), "nt": c.nt, "nfreq": int(c.freqs.size),
           "l2": "inputs larger than L2 (16 GB transforms, 425 MB residuals); no flush"}
    if extra:
        cfg.update(extra)
    return cfg


def gram_roofline(precision, nr, nf, npts, c, ms, peak, kind):
    """The Gram kernel against the tensor peak (mixed) or as FP32 CUDA-core work (fp32).  Issued
    tensor work: 64-receiver panel pairs on and above the diagonal, each 128 x 128 x G per
    frequency (G: the grid sum's length at the device pitch), 3 bf16 products (hi hi, hi lo,
    lo hi).  Algorithmic work: the Hermitian half of the complex Gram over the padded grid's
    Nx = NZ x NX points, 8 Nf Nr^2 Nx (Nr + 1) / (2 Nr) real flops, against the bf16 peak and
    against the bf16x3 rate (a third of it: three products per flop of the FP32-class result)."""
    NZ, NX = c.nz + 2 * c.nsponge, c.nx + 2 * c.nsponge
    PX = max(64, -(-(NX + 4) // 64) * 64)  # row pitch of the device levels
    G = -(-(NZ * PX) // 256) * 256  # padded point count the Gram sums over
    Nx = NZ * NX
    n64 = -(-nr // 64)
    issued = n64 * (n64 + 1) / 2 * 128 * 128 * 2 * 3 * G * nf
    alg = 8.0 * nf * nr * nr * Nx * (nr + 1) / (2 * nr)
    alg_tf = alg / (ms * 1e-3) / 1e12
    out = {"kernel": "k_gram_tc (bf16x3 tcgen05 Gram)" if precision == "mixed" else "k_gram_partial (FP32)",
           "ms": ms, "algorithmic_tflops": alg_tf, "algorithmic_flops": alg, "nx_points": Nx}
    if precision == "mixed":
        out.update({"bound": "tensor", "achieved": issued / (ms * 1e-3) / 1e12, "peak": peak,
                    "peak_kind": kind, "unit": "TFLOP/s", "frac": issued / (ms * 1e-3) / 1e12 / peak,
                    "algorithmic_frac_of_bf16": alg_tf / peak,
                    "algorithmic_frac_of_bf16x3": alg_tf / (peak / 3.0),
                    "note": "achieved = issued bf16 MMA flops (3 products, padded panels and pitch) / "
                            "kernel time (CUDA events around the launch inside egh_hessian); "
                            "algorithmic = Hermitian half over the Nx grid points"})
    return out


def variants_bench(torch, egh, ctx, c, v_start, resid, mult, stream, ev):
    """The paper's cheaper forms on the benchmark workload, after the timed steps (not part of
    the headline): Green functions of a band-limited source with the transform decimated 10x in
    time (its Hessian against the Dirac one), the diagonal-Hessian deblur, and a Hessian of 100
    receivers drawn one per subset."""
    import numpy as np

    import synth

    def timed(fn):
        e0, e1 = ev(), ev()
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    Qd = ctx.get_hessian(False)
    w = synth.ricker(250, c.dt, 8.0, t0=0.125).astype(np.float32)
    decim = 10
    ctx.green_bandlimited(v_start, w, decim)  # untimed: captures the decimated chunks' graphs
    g_ms = timed(lambda: ctx.green_bandlimited(v_start, w, decim))
    st = ctx.stats()
    ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
    Qb = ctx.get_hessian(False)
    err = [float(np.linalg.norm(Qb[k] - Qd[k]) / np.linalg.norm(Qd[k])) for k in range(Qd.shape[0])]
    diag_ms = timed(lambda: ctx.deblur_diag(resid, mult))
    sel = egh.sample_receivers(c.rec_ix.size, 100, seed=2025, iteration=0)
    with egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz[sel],
                     c.rec_ix[sel], c.freqs, precision=egh.EGH_PREC_MIXED) as c100:
        # first pass untimed: it includes the one-off tuning of the FD rows and the Gram split
        c100.green(v_start)
        c100.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        c100.factor()
        sub_green = timed(lambda: c100.green(v_start))
        sub_hf = timed(lambda: (c100.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha), c100.factor()))
    return {
        "bandlimited_decimated": {
            "wavelet": "Ricker 8 Hz, 250 samples", "decim": decim, "green_ms": g_ms,
            "green_fd_ms": st["fd_ms"], "green_transform_ms": st["dft_ms"],
            "hessian_rel_err_vs_dirac_max": max(err), "hessian_rel_err_vs_dirac_min": min(err)},
        "diagonal_hessian_deblur_ms": diag_ms,
        "random_receivers_100": {"green_ms": sub_green, "hessian_factor_ms": sub_hf,
                                 "receivers": "one per subset of 231, SplitMix64 seed 2025"},
    }


def serve_bench(torch, egh, precision, requests=240, seed=11):
    """Serving form: Poisson-arriving deblur requests against 4 resident factored Hessian sets
    (Nr 101/211/331/461, Nf 20/27/33/40, 2-10 Hz; seeded synthetic Hermitian positive-definite
    Q_k = A A^H / m + 0.05 mean diag I); each request U{1..64} sources, nt U{2000..4000}, FP32
    band-limited (2-10 Hz) seeded Gaussian residuals from pinned host memory, results back to
    pinned host memory.  The arrival rate is 70% of the throughput measured with all requests
    queued at once.  Returns p50/p99 latency and sources/s."""
    import numpy as np

    import synth

    rng = np.random.default_rng(seed)
    shapes = ((101, 20), (211, 27), (331, 33), (461, 40))
    dt, max_nt = 1e-3, 4096
    with egh.Server(24 << 30, slots=6, max_batch_sources=128, precision=precision) as sv:
        ids, sets_host = [], []
        for nrec, nf in shapes:
            A = torch.randn((nf, nrec, 2 * nrec), dtype=torch.complex64, device="cuda",
                            generator=torch.Generator(device="cuda").manual_seed(seed + nrec))
            Q = A @ A.conj().transpose(1, 2) / (2 * nrec)
            mu = 0.05 * torch.diagonal(Q, dim1=1, dim2=2).real.mean()
            Q = (Q + mu * torch.eye(nrec, device="cuda")).cpu().numpy()
            ids.append(sv.add_set(Q, np.linspace(2.0, 10.0, nf), dt, 4000, max_nt))
            sets_host.append((Q, np.linspace(2.0, 10.0, nf), dt, 4000))
        # a pool of pinned buffers, one per request in flight at most
        pool = 8
        maxb = 64 * 461 * 4000
        ins = [torch.empty(maxb, dtype=torch.float32, pin_memory=True) for _ in range(pool)]
        outs = [torch.empty(maxb, dtype=torch.float32, pin_memory=True) for _ in range(pool)]
        base = torch.from_numpy(
            synth.bandlimited_noise(rng, (461, 4000), dt, 2.0, 10.0).astype(np.float32).reshape(-1))
        for b in ins:
            b.view(64, -1).copy_(base.expand(64, -1))
        spec = [(int(rng.integers(4)), int(rng.integers(1, 65)), int(rng.integers(2000, 4001)))
                for _ in range(requests)]

        def run(arrivals):
            sv.reset_stats()
            live = []
            t0 = time.perf_counter()
            for i, (sid, ns, nt_d) in enumerate(spec):
                if arrivals is not None:
                    while time.perf_counter() - t0 < arrivals[i]:
                        pass
                if len(live) == pool:
                    sv.wait(live.pop(0)[0])
                slot = i % pool
                shape = (ns, shapes[sid][0], nt_d)
                n = ns * shapes[sid][0] * nt_d
                rid = sv.submit(ids[sid], ins[slot][:n].view(shape), outs[slot][:n].view(shape))
                live.append((rid, slot))
            for rid, _ in live:
                sv.wait(rid)
            return sv.stats()

        run(None)                       # warm-up (launch paths, arena)
        full = run(None)                # all requests queued at once: capacity
        srcs = sum(s[1] for s in spec)
        rate = 0.7 * full["completed"] / full["span_s"]
        gaps = rng.exponential(1.0 / rate, size=requests)
        st = run(np.cumsum(gaps) - gaps[0])
        # a seeded sample of requests of the two smaller sets, kept (inputs, results, Hessians)
        # for the check against the FP64 oracle in the cpu_baseline leg
        samples = []
        for sid, ns, nt_d in [(0, 3, 2400), (1, 2, 3100), (0, 17, 2000), (1, 5, 4000)]:
            nr = shapes[sid][0]
            r = synth.bandlimited_noise(rng, (ns, nr, nt_d), dt, 2.0, 10.0).astype(np.float32)
            rin = torch.from_numpy(r).pin_memory()
            out = torch.empty_like(rin).pin_memory()
            sv.wait(sv.submit(ids[sid], rin, out))
            samples.append({"set": sid, "resid": r, "mult": out.numpy().copy()})
    return {"workload": "4 resident Hessian sets Nr 101/211/331/461, Nf 20/27/33/40 (synthetic HPD "
                        "A A^H/m + 0.05 mean diag I), Poisson arrivals at 70% of capacity, "
                        f"{requests} requests of U{{1..64}} sources x nt U{{2000..4000}}",
            "precision": "mixed" if precision == egh.EGH_PREC_MIXED else "fp32",
            "sources_per_s": st["sources_done"] / st["span_s"],
            "p50_ms": st["p50_s"] * 1e3, "p99_ms": st["p99_s"] * 1e3, "mean_ms": st["mean_s"] * 1e3,
            "arrival_rate_per_s": rate, "capacity_sources_per_s": srcs / full["span_s"],
            "batches": st["batches"], "requests": st["completed"],
            "peak_in_flight": st["peak_in_flight"], "peak_arena_bytes": st["peak_bytes_in_use"],
            "_sets": sets_host, "_samples": samples}


def salt_bench(torch, egh, precision, ev, stream, steps=1, warmup=1):
    """The batched form (three patches of the 1701x351 salt model, 161/257/341 receivers, nt 6000,
    40 frequencies 2-10 Hz each, all 120 Hessians factored in one persistent launch under a CUDA
    graph), as a leg of the default run: update seconds, the batched factorisation, and the Green
    stage's rate on 12 B per receiver point-step."""
    import numpy as np

    import synth

    c = synth.case_salt_patches()
    prec = egh.EGH_PREC_MIXED if precision == "mixed" else egh.EGH_PREC_FP32
    v = torch.from_numpy(np.float32(c.vel_true)).cuda()
    ctxs = [egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt,
                        np.zeros(p.size, np.int32), p, c.freqs, precision=prec) for p in c.patches]
    batch = egh.Batch(ctxs)
    try:
        def step():
            e = [ev() for _ in range(3)]
            e[0].record(stream)
            for ctx in ctxs:
                ctx.green(v)
                ctx.hessian(egh.EGH_MU_REL_MEANDIAG, 1e-2)
                ctx.release_green()
            e[1].record(stream)
            batch.factor()
            e[2].record(stream)
            torch.cuda.synchronize()
            return e[0].elapsed_time(e[2]) / 1e3, e[1].elapsed_time(e[2])

        for _ in range(warmup):
            step()
        res = [step() for _ in range(steps)]
        ps = sum(ctx.stats()["point_steps"] for ctx in ctxs)
        upd = statistics.mean(r[0] for r in res)
        fac = statistics.mean(r[1] for r in res)
        hbm, _ = _peaks()
        gs = 12.0 * ps / (upd - fac / 1e3) / 1e9
        return {"workload": "salt 1701x351 (padded 1741x391), three patches of 161/257/341 receivers, "
                            "nt 6000, 40 frequencies 2-10 Hz each, mu 1e-2 mean diag",
                "precision": precision, "update_build_factor_s": upd, "batched_factor_ms": fac,
                "hessians": 120, "green_and_hessian_gbs": gs, "green_and_hessian_frac": gs / hbm,
                "note": "Green stage + Hessians per patch (Green buffers released after each), then "
                        "the 120 Hessians factored in one persistent launch (CUDA graph); "
                        "12 B per receiver point-step"}
    finally:
        batch.close()
        for ctx in ctxs:
            ctx.close()


def run_salt(args):
    """Batched form on the salt workload: three surface patches (161, 257, 341 receivers) of the
    1701x351 model, 40 frequencies 2-10 Hz each, nt 6000.  One step = each patch's Green
    functions and Hessians (its Green-stage buffers released after egh_hessian) and then all
    120 Hessians factored in one persistent launch replayed as a CUDA graph."""
    import numpy as np
    import torch

    import synth
    from paper_2512_16642_gb300 import egh

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    c = synth.case_salt_patches()
    prec = egh.EGH_PREC_MIXED if args.precision == "mixed" else egh.EGH_PREC_FP32
    v = torch.from_numpy(np.float32(c.vel_true)).cuda()
    ctxs = [egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt,
                        np.zeros(p.size, np.int32), p, c.freqs, precision=prec) for p in c.patches]
    stream = torch.cuda.current_stream()
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    batch = egh.Batch(ctxs)

    def step():
        e = [ev() for _ in range(3)]
        e[0].record(stream)
        for ctx in ctxs:
            ctx.green(v)
            ctx.hessian(egh.EGH_MU_REL_MEANDIAG, 1e-2)
            ctx.release_green()
        e[1].record(stream)
        batch.factor()
        e[2].record(stream)
        torch.cuda.synchronize()
        return e[0].elapsed_time(e[2]), e[1].elapsed_time(e[2])

    for _ in range(args.warmup):
        step()
    _barrier(ws)
    clk = ClockSampler(local)
    clk.start()
    l0 = ctxs[0].stats()["kernel_launches"]
    res = [step() for _ in range(args.steps)]
    torch.cuda.synchronize()
    _barrier(ws)
    clocks = clk.stop()
    launches = ctxs[0].stats()["kernel_launches"] - l0
    total = statistics.mean(r[0] for r in res) / 1e3
    fac = statistics.mean(r[1] for r in res)
    ps = sum(ctx.stats()["point_steps"] for ctx in ctxs)
    total_max = _max_over_ranks(ws, total)  # every rank takes part in the reduction
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": total_max / ws, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_max * 1e3,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "salt 1701x351 (padded 1741x391), dx 10 m, three surface patches of "
                                   "161/257/341 receivers, nt 6000 dt 1 ms, 40 frequencies 2-10 Hz each, "
                                   "mu 1e-2 mean diag; 120 Hessians factored in one persistent launch "
                                   "(CUDA graph)", "precision": args.precision,
                       "l2": "inputs larger than L2; no flush"},
            "stages_ms": {"green_and_hessians": total * 1e3 - fac, "batched_factor": fac},
            "green_stage": {"achieved": 12.0 * ps / (total - fac / 1e3) / 1e9, "unit": "GB/s",
                            "note": "12 B per receiver point-step over Green + Hessian time"},
            "gpu_launches": int(launches), "clocks": clocks}), flush=True)
    batch.close()
    for ctx in ctxs:
        ctx.close()


def run_reference(args):
    import synth

    ws, rank, _ = _dist()
    if rank != 0:
        return
    c = synth.case_layered()
    for _ in range(args.warmup):
        oracle_sample(c, green_steps=20, deblur_sources=1)
    vals, ms = [], []
    last = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        last = oracle_sample(c)
        ms.append((time.perf_counter() - t0) * 1e3)
        vals.append(last["build_factor_s"])
    v = statistics.mean(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.mean(ms),
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": _workload(c, {"sample": last["sample"]}),
        "deblur_sources_per_s": last["sources_per_s"],
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": last["cores"], "kind": "oracle",
                         "sample": last["sample"]},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import numpy as np
    import torch

    import synth
    from paper_2512_16642_gb300 import egh

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    c = synth.case_layered()
    if args.slice:
        c = synth.slice_case(c, nrec=args.slice_receivers, nt=args.slice_nt)
        args.e2e_steps, args.no_cpu_baseline = 0, True
    nr, ns, nt, nf = c.rec_ix.size, c.src_ix.size, c.nt, c.freqs.size
    ctx = egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz, c.rec_ix, c.freqs,
                      dft_chunk=args.dft_chunk, fd_kernel=args.fd_kernel,
                      precision=egh.EGH_PREC_MIXED if args.precision == "mixed" else egh.EGH_PREC_FP32)
    stream = torch.cuda.current_stream()
    v_start = torch.from_numpy(np.float32(c.vel_start)).cuda()
    if args.resid == "noise":
        noise = synth.bandlimited_noise(np.random.default_rng(5), (ns, nr, nt), c.dt, 2.0, 10.0)
        resid = torch.from_numpy(noise.astype(np.float32)).cuda()
    else:
        v_true = torch.from_numpy(np.float32(c.vel_true)).cuda()
        w32 = synth.ricker(nt, c.dt, c.ricker_hz).astype(np.float32)
        resid = torch.empty((ns, nr, nt), device="cuda")
        tmp = torch.empty_like(resid)
        ctx.forward(v_true, c.src_iz, c.src_ix, w32, resid)
        ctx.forward(v_start, c.src_iz, c.src_ix, w32, tmp)
        resid -= tmp
        del tmp
    mult = torch.empty_like(resid)

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(rec=None):
        e = [ev() for _ in range(4)]
        e[0].record(stream)
        ctx.green(v_start)
        if rec is not None:
            st_g = ctx.stats()
            kern.append((st_g["fd_ms"], st_g["fd_launches"], st_g["dft_ms"], st_g["dft_launches"]))
        e[1].record(stream)
        ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        if rec is not None:
            gram_ms.append(ctx.stats()["gram_ms"])
        ctx.factor()
        e[2].record(stream)
        ctx.deblur(resid, mult)
        e[3].record(stream)
        if rec is not None:
            rec.append(e)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    l0 = ctx.stats()["kernel_launches"]
    recs, kern, gram_ms = [], [], []
    t_start, t_end = ev(), ev()
    t_start.record(stream)
    for _ in range(args.steps):
        step(recs)
    t_end.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctx.stats()["kernel_launches"] - l0
    total_ms = t_start.elapsed_time(t_end)
    refinement = None
    if args.precision == "mixed":
        cb, rf = ctx.get_refinement()
        refinement = {"threshold": 1e4, "refined_frequencies": int(rf.sum()), "of": int(rf.size),
                      "cond_bound_min": float(cb.min()), "cond_bound_max": float(cb.max()),
                      "note": "solves of a frequency get one refinement step when its condition "
                              "bound (||Q||_F over the smaller of mu and a power estimate of "
                              "lambda_min) exceeds the threshold"}
    green_ms = [e[0].elapsed_time(e[1]) for e in recs]
    bf_ms = [e[0].elapsed_time(e[2]) for e in recs]
    deb_ms = [e[2].elapsed_time(e[3]) for e in recs]
    bf_s = statistics.mean(bf_ms) / 1e3
    bf_s_max = _max_over_ranks(ws, bf_s)
    ms_step = _max_over_ranks(ws, total_ms / args.steps)
    st = ctx.stats()

    # end to end through the same entry points with pinned host buffers
    v_host = torch.from_numpy(np.float32(c.vel_start)).pin_memory()
    r_host = resid.cpu().pin_memory()
    m_host = torch.empty_like(r_host).pin_memory()
    e2e_bf, e2e_deb, e2e_deb_dev = [], [], []
    for i in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.green(v_host)
        ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        ctx.factor()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        d0, d1 = ev(), ev()
        d0.record(stream)
        ctx.deblur(r_host, m_host)
        d1.record(stream)
        t2 = time.perf_counter()
        if i > 0:
            e2e_bf.append(t1 - t0)
            e2e_deb.append(t2 - t1)
            torch.cuda.synchronize()
            e2e_deb_dev.append(d0.elapsed_time(d1))
    e2e_v = _max_over_ranks(ws, statistics.mean(e2e_bf)) / ws if e2e_bf else None

    if rank != 0:
        return
    hbm, peak_kind = _peaks()
    tc_peak, tc_kind = _bf16_peak()
    point_steps = st["point_steps"]
    green_s = statistics.mean(green_ms) / 1e3
    with open(os.path.join(ROOT, "paper_2512_16642_gb300", "csrc", "fd.cu"), "rb") as f:
        fd_sha = hashlib.sha256(f.read()).hexdigest()
    traffic_ok = KERNEL_TRAFFIC["fd_sha256"] == fd_sha
    with open(os.path.join(ROOT, "paper_2512_16642_gb300", "csrc", "gram_tc.cu"), "rb") as f:
        gram_traffic = (KERNEL_TRAFFIC["k_gram_tc"].get(st["gram_splits"])
                        if KERNEL_TRAFFIC["gram_sha256"] == hashlib.sha256(f.read()).hexdigest()
                        and args.precision == "mixed" and nr == 231 else None)
    fd_ms = statistics.mean(k[0] for k in kern)
    fd_n = kern[-1][1]
    dft_ms = statistics.mean(k[2] for k in kern)
    dft_n = kern[-1][3]
    npts = point_steps // (nr * nt)  # padded grid points NZ * NX
    nchunk = dft_n // ((nr + st["batch_receivers"] - 1) // st["batch_receivers"])
    # FD step: 12 algorithmic bytes per receiver point-step (read u^n, u^{n-1}, write u^{n+1})
    fd_alg = 12.0 * point_steps / fd_n
    fd_achieved = fd_alg / (fd_ms / fd_n * 1e-3) / 1e9
    # transform: 4 B per receiver point-step (bf16 hi + lo snapshot) + the gh read-modify-write
    # of 2 nf floats per receiver point per chunk (write only for the first chunk)
    dft_alg = (4.0 * point_steps + nr * npts * 2 * nf * 4 * (2 * nchunk - 1)) / dft_n
    dft_achieved = dft_alg / (dft_ms / dft_n * 1e-3) / 1e9
    serving = None
    if not args.slice and not args.no_serving:
        serving = serve_bench(torch, egh, egh.EGH_PREC_MIXED if args.precision == "mixed"
                              else egh.EGH_PREC_FP32)
    # the other Hessian arithmetic on the same transforms, for comparison (not the headline)
    other = {}
    if not args.slice:
        alt = egh.EGH_PREC_FP32 if args.precision == "mixed" else egh.EGH_PREC_MIXED
        with egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz,
                         c.rec_ix, c.freqs, precision=alt, dft_chunk=args.dft_chunk) as ctx2:
            ctx2.green(v_start)
            hf = []
            for _ in range(2):
                e0, e1 = ev(), ev()
                e0.record(stream)
                ctx2.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
                ctx2.factor()
                e1.record(stream)
                torch.cuda.synchronize()
                hf.append(e0.elapsed_time(e1))
            other = {"precision": "fp32" if alt == egh.EGH_PREC_FP32 else "mixed",
                     "hessian_factor_ms": min(hf)}
            # the whole update in the other arithmetic (Green stage, Hessians, factors, deblur)
            m2 = torch.empty_like(resid)
            e = [ev() for _ in range(4)]
            e[0].record(stream)
            ctx2.green(v_start)
            e[1].record(stream)
            ctx2.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
            ctx2.factor()
            e[2].record(stream)
            ctx2.deblur(resid, m2)
            e[3].record(stream)
            torch.cuda.synchronize()
            other.update({"update_build_factor_s": e[0].elapsed_time(e[2]) / 1e3,
                          "green_ms": e[0].elapsed_time(e[1]), "deblur_ms": e[2].elapsed_time(e[3]),
                          "deblur_sources_per_s": ns / (e[2].elapsed_time(e[3]) / 1e3),
                          "mult_rel_diff_vs_headline": float((m2 - mult).norm() / mult.norm())})
            del m2
    variants = None
    if not args.slice and not args.no_serving:
        variants = variants_bench(torch, egh, ctx, c, v_start, resid, mult, stream, ev)
    batched = None
    if not args.slice and not args.no_batched and ws == 1:
        ctx.close()  # the salt workload's largest patch needs the device memory
        torch.cuda.empty_cache()
        batched = salt_bench(torch, egh, args.precision, ev, stream)
    line = {
        "metric": METRIC, "value": bf_s_max / ws, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32/bf16x3" if args.precision == "mixed" else "f32/bf16x3-transform",
        "data": "synthetic",
        "config": _workload(c, {"batch_receivers": st["batch_receivers"], "dft_chunk": st["dft_chunk"],
                                "gram_splits": st["gram_splits"], "fd_rows": st["fd_rows"], "fd_kernel": st["fd_kernel"],
                                "precision": args.precision,
                                "residuals": "forward modelling (true - start)" if args.resid == "model"
                                else "seeded band-limited noise 2-10 Hz"}),
        "stages_ms": {"green": statistics.mean(green_ms), "green_fd": fd_ms, "green_transform": dft_ms,
                      "build_factor": statistics.mean(bf_ms),
                      "hessian_factor": statistics.mean(bf_ms) - statistics.mean(green_ms),
                      "deblur": statistics.mean(deb_ms)},
        "deblur_sources_per_s": ns / (statistics.mean(deb_ms) / 1e3),
        "refinement": refinement,
        "other_precision": other or None,
        "serving": serving,
        "variants": variants,
        "roofline": {"kernel": "k_fd_step (FD step, 99% of the update's stream time)", "bound": "hbm",
                     "achieved": fd_achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": fd_achieved / hbm,
                     "traffic": KERNEL_TRAFFIC["k_fd_step"] if traffic_ok else None,
                     "algorithmic_bytes_per_launch": fd_alg,
                     "launches": fd_n, "avg_launch_ms": fd_ms / fd_n,
                     "note": "12 B per receiver point-step; duration = per-chunk CUDA events on the FD "
                             "stream / launches (graph-replayed steps, gaps included); the measured "
                             "limiter is L2 bandwidth (see profiles/)"},
        "roofline_transform": {"kernel": "k_dft_tc (tensor-core transform)", "bound": "hbm",
                               "achieved": dft_achieved, "peak": hbm, "peak_kind": peak_kind,
                               "unit": "GB/s", "frac": dft_achieved / hbm,
                               "traffic": KERNEL_TRAFFIC["k_dft_tc"] if traffic_ok else None,
                               "algorithmic_bytes_per_launch": dft_alg, "launches": dft_n,
                               "avg_launch_ms": dft_ms / dft_n,
                               "note": "runs beside the next chunk's FD steps on a low-priority stream"},
        "roofline_gram": dict(gram_roofline(args.precision, nr, nf, npts, c, statistics.mean(gram_ms),
                                            tc_peak, tc_kind), traffic=gram_traffic),
        "green_stage": {"achieved": 12.0 * point_steps / green_s / 1e9, "unit": "GB/s",
                        "frac": 12.0 * point_steps / green_s / 1e9 / hbm,
                        "note": "whole egh_green (FD + transform), 12 B per receiver point-step"},
        "e2e": None if e2e_v is None else {
                "value": e2e_v, "unit": UNIT,
                "h2d_bytes_per_step": int(v_host.numel() * 4 + r_host.numel() * 4),
                "d2h_bytes_per_step": int(m_host.numel() * 4 + 8 + 4 * nf),
                "deblur_sources_per_s": ns / statistics.median(e2e_deb),
                "deblur_ms": [round(t * 1e3, 3) for t in e2e_deb],
                # the same calls on the stream's clock: copies + kernels, without the host's share
                "deblur_stream_ms": [round(t, 3) for t in e2e_deb_dev],
                "note": "green from pinned host velocity + hessian + factor; deblur from pinned host "
                        "residuals to pinned host multipliers"},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if not args.no_cpu_baseline and ws == 1:
        ob = oracle_sample(c)
        line["cpu_baseline"] = {"value": ob["build_factor_s"], "unit": UNIT, "cores": ob["cores"],
                                "kind": "oracle", "sample": ob["sample"],
                                "deblur_sources_per_s": ob["sources_per_s"]}
        if serving is not None:
            errs = serving_error(serving)
            serving["rel_err_vs_oracle"] = errs
            serving["max_rel_err_vs_oracle"] = max(errs)
            serving["error_note"] = ("multipliers of 4 kept requests (sets of 101 and 211 receivers) "
                                     "against the FP64 oracle; tolerance 1e-3")
    if serving is not None:
        serving.pop("_sets", None)
        serving.pop("_samples", None)
    if batched is not None:
        line["batched"] = batched
    print(json.dumps(line), flush=True)


def run_sharded(args):
    """One model update of the layered workload split over the ranks (strong scaling): each rank
    solves its block of receivers, one exchange moves the transforms to frequency blocks, the
    penalty comes from one all-reduce, each rank factors and deblurs its frequencies and the
    multipliers are summed over the ranks (paper_2512_16642_gb300.sharded).  value = build +
    factor seconds per update (Green solves, exchange, Hessians, penalty, factorisation), the max
    over ranks; the deblur and the end-to-end update from pinned host buffers ride along."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import synth
    from paper_2512_16642_gb300 import egh, sharded

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    c = synth.case_layered()
    if args.slice:
        c = synth.slice_case(c, nrec=args.slice_receivers, nt=args.slice_nt)
        args.e2e_steps = 0
    nr, ns, nt, nf = c.rec_ix.size, c.src_ix.size, c.nt, c.freqs.size
    geom = {k: c[k] for k in ("nz", "nx", "dz", "dx", "nsponge", "sponge_R", "dt", "nt", "rec_iz",
                              "rec_ix", "freqs")}
    prec = egh.EGH_PREC_MIXED if args.precision == "mixed" else egh.EGH_PREC_FP32
    shard = sharded.Shard(geom, rank, ws, precision=prec, dft_chunk=args.dft_chunk)
    stream = torch.cuda.current_stream()
    vel = torch.from_numpy(np.float32(c.vel_start)).cuda()
    noise = synth.bandlimited_noise(np.random.default_rng(5), (ns, nr, nt), c.dt, 2.0, 10.0)
    resid = torch.from_numpy(noise.astype(np.float32)).cuda()
    mult = torch.empty_like(resid)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def step(v, r, m):
        e = [ev() for _ in range(3)]
        e[0].record(stream)
        sends = shard.green(v)
        recvs = shard.receive_buffers()
        if ws > 1:
            sharded.exchange(sends, recvs, rank)
        else:
            recvs[0].copy_(sends[0])
        shard.assemble(recvs)
        d = torch.tensor([shard.hessian()], dtype=torch.float64, device="cuda")
        if ws > 1:
            dist.all_reduce(d)
        shard.factor(float(d.item()), c.mu_alpha)
        e[1].record(stream)
        shard.deblur(r, m)
        if ws > 1:
            dist.all_reduce(m)
        e[2].record(stream)
        return e

    for _ in range(args.warmup):
        step(vel, resid, mult)
    torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    ctxs = [x for x in (shard.green_ctx, shard.hess_ctx) if x is not None]
    l0 = ctxs[0].stats()["kernel_launches"]
    t0, t1 = ev(), ev()
    t0.record(stream)
    recs = [step(vel, resid, mult) for _ in range(args.steps)]
    t1.record(stream)
    torch.cuda.synchronize()
    _barrier(ws)
    torch.cuda.synchronize()
    clocks = clk.stop()
    launches = ctxs[0].stats()["kernel_launches"] - l0
    bf = statistics.mean(e[0].elapsed_time(e[1]) for e in recs) / 1e3
    deb = statistics.mean(e[1].elapsed_time(e[2]) for e in recs)
    bf_max = _max_over_ranks(ws, bf)
    ms_step = _max_over_ranks(ws, t0.elapsed_time(t1) / args.steps)
    # end to end from pinned host buffers: the velocity and residuals copied in, the multipliers
    # copied out, inside the timed span
    e2e = None
    if args.e2e_steps > 0:
        v_host = torch.from_numpy(np.float32(c.vel_start)).pin_memory()
        r_host = resid.cpu().pin_memory()
        m_host = torch.empty_like(r_host).pin_memory()
        times = []
        for i in range(args.e2e_steps + 1):
            torch.cuda.synchronize()
            _barrier(ws)
            a = time.perf_counter()
            vel.copy_(v_host, non_blocking=True)
            resid.copy_(r_host, non_blocking=True)
            step(vel, resid, mult)
            m_host.copy_(mult, non_blocking=True)
            torch.cuda.synchronize()
            if i > 0:
                times.append(time.perf_counter() - a)
        e2e_v = _max_over_ranks(ws, statistics.mean(times))
        e2e = {"value": e2e_v, "unit": UNIT, "h2d_bytes_per_step": int(v_host.numel() * 4 + r_host.numel() * 4),
               "d2h_bytes_per_step": int(m_host.numel() * 4),
               "note": "whole sharded update (build, factor and deblur) per rank from pinned host "
                       "velocity and residuals to pinned host multipliers, max over ranks"}
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": bf_max, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": False,
            "scaling": "strong", "vs_baseline": None,
            "dtype": "f32/bf16x3" if args.precision == "mixed" else "f32/bf16x3-transform",
            "data": "synthetic",
            "config": _workload(c, {"precision": args.precision, "parallelism": f"sharded{ws}",
                                    "receiver_blocks": shard.rb, "frequency_blocks": shard.kb,
                                    "residuals": "seeded band-limited noise 2-10 Hz"}),
            "stages_ms": {"build_factor": bf * 1e3, "deblur": deb},
            "deblur_sources_per_s": ns / (deb / 1e3),
            "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks}), flush=True)
    shard.close()


def run_deblur(args):
    """The deblur kernels alone at the layered workload's shape (231 receivers, 26 frequencies
    3.0:0.2:8.0 Hz, 115 sources x 4000 samples), through a serving set so that no Green stage
    runs: a seeded synthetic Hermitian positive-definite Hessian set (Q_k = A A^H / m + 0.05 mean
    diag I) and band-limited noise residuals from pinned host memory.  Prints one JSON line with
    the request latency (host copies included) for profiling captures; not the benchmark."""
    import numpy as np
    import torch

    import synth
    from paper_2512_16642_gb300 import egh

    rng = np.random.default_rng(3)
    n, nf, ns, nt = 231, 26, 115, 4000
    A = (rng.standard_normal((nf, n, 2 * n)) + 1j * rng.standard_normal((nf, n, 2 * n))) / np.sqrt(2 * n)
    Q = A @ A.conj().transpose(0, 2, 1)
    Q += 0.05 * np.mean(np.einsum("kii->ki", Q).real) * np.eye(n)
    Q = (0.5 * (Q + Q.conj().transpose(0, 2, 1))).astype(np.complex64)
    f = np.round(np.arange(3.0, 8.0 + 1e-9, 0.2), 6)
    r = synth.bandlimited_noise(rng, (ns, n, nt), 1e-3, 3.0, 8.0)
    prec = egh.EGH_PREC_MIXED if args.precision == "mixed" else egh.EGH_PREC_FP32
    lat = []
    with egh.Server(8 << 30, slots=2, max_batch_sources=ns, precision=prec) as sv:
        sid = sv.add_set(Q, f, 1e-3, nt, nt)
        rin = torch.from_numpy(np.ascontiguousarray(r, np.float32)).pin_memory()
        out = torch.empty_like(rin).pin_memory()
        for _ in range(max(1, args.steps)):
            lat.append(sv.wait(sv.submit(sid, rin, out)))
    print(json.dumps({"workload": "deblur kernels alone, layered shape (231 receivers, 26 frequencies, "
                                  "115 sources x 4000 samples), synthetic HPD Hessians",
                      "precision": args.precision, "latency_s": lat}), flush=True)


def main():
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "salt":
        run_salt(args)
    elif args.workload == "deblur":
        run_deblur(args)
    elif args.sharded or int(os.environ.get("WORLD_SIZE", "1")) > 1:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
