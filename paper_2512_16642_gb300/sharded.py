"""Sharded model update across GPUs: one process (rank) per GPU, collectives through
torch.distributed (NCCL on GPUs).

The Green-function solves are independent per receiver and each frequency's Hessian and
factorisation are independent of the others (Algorithm 2: one solve per active receiver, then an
inversion per frequency), so one update splits as:

  1. rank r solves the receivers of its block R_r at every frequency (a context holding R_r);
  2. one all-to-all exchange: rank r sends the transforms of R_r at the frequencies K_q to rank q,
     which assembles all receivers at its frequencies K_q (a context holding every receiver and
     K_q, filled by egh_import_green);
  3. each rank forms its Hessians without the penalty; the penalty mu = alpha x mean diagonal needs
     the sum of the ranks' diagonal sums: one all-reduce of a scalar;
  4. each rank sets mu and factors its frequencies;
  5. each rank deblurs the (replicated) residuals at its frequencies with the synthesis weights of
     the full frequency list; the multipliers are the sum over ranks (one all-reduce), since the
     synthesis back to time is a sum over frequencies.

Blocks are contiguous and their sizes differ by at most one.  Each step of the path runs in the
library's kernels through `Context`; this module holds only the partitioning and the exchange.
`context_factory` builds a rank's contexts: the library's `egh.Context` by default; any object
with the same methods serves (the CPU tests pass one backed by another implementation).
"""
from __future__ import annotations

import numpy as np

from . import egh


def block(n: int, parts: int, i: int) -> tuple[int, int]:
    """[begin, end) of part i when n items are split into `parts` contiguous blocks."""
    base, extra = divmod(n, parts)
    b = i * base + min(i, extra)
    return b, b + base + (1 if i < extra else 0)


class Shard:
    """One rank's share of a sharded update.

    geom: dict with nz, nx, dz, dx, nsponge, sponge_R, dt, nt, rec_iz, rec_ix, freqs (the whole
    survey); context keywords (precision, gram_splits, dft_chunk, ...) pass through to both
    contexts.  Receivers R = block(nrec, world, rank), frequencies K = block(nf, world, rank).
    """

    def __init__(self, geom, rank: int, world: int, context_factory=None, **ctx_kw):
        self.rank, self.world = rank, world
        self.g = geom
        self.nrec = len(geom["rec_ix"])
        self.freqs = np.asarray(geom["freqs"], dtype=np.float64)
        self.nf = self.freqs.size
        make = context_factory or egh.Context
        self.rb = [block(self.nrec, world, r) for r in range(world)]
        self.kb = [block(self.nf, world, q) for q in range(world)]
        r0, r1 = self.rb[rank]
        k0, k1 = self.kb[rank]
        common = (geom["nz"], geom["nx"], geom["dz"], geom["dx"], geom["nsponge"], geom["sponge_R"],
                  geom["dt"], geom["nt"])
        rec_iz = np.asarray(geom["rec_iz"], np.int32)
        rec_ix = np.asarray(geom["rec_ix"], np.int32)
        self.green_ctx = (make(*common, rec_iz[r0:r1], rec_ix[r0:r1], self.freqs, **ctx_kw)
                          if r1 > r0 else None)
        self.hess_ctx = (make(*common, rec_iz, rec_ix, self.freqs[k0:k1], **ctx_kw)
                         if k1 > k0 else None)
        if self.hess_ctx is not None:
            self.hess_ctx.set_synthesis_frequencies(self.freqs, k0)
        self.mu = None

    # -- step 1: the rank's receivers at every frequency, cut by destination frequency block
    def green(self, vel):
        """Solves this rank's receivers; returns the send buffers, one per destination rank q:
        the transforms of this rank's receivers at q's frequencies."""
        r0, r1 = self.rb[self.rank]
        sends = []
        for q in range(self.world):
            k0, k1 = self.kb[q]
            sends.append(self._buffer(r1 - r0, k1 - k0))
        if self.green_ctx is not None:
            self.green_ctx.green(vel)
            for q in range(self.world):
                k0, k1 = self.kb[q]
                if k1 > k0:
                    self.green_ctx.export_green(k0, k1 - k0, sends[q])
        return sends

    def receive_buffers(self):
        """One buffer per source rank r: r's receivers at this rank's frequencies."""
        k0, k1 = self.kb[self.rank]
        return [self._buffer(r1 - r0, k1 - k0) for r0, r1 in self.rb]

    # -- step 2 (receiving side): all receivers at this rank's frequencies
    def assemble(self, recvs):
        if self.hess_ctx is None:
            return
        import torch

        parts = [b for b in recvs if b.numel()]
        self.hess_ctx.import_green(torch.cat(parts, dim=0) if len(parts) > 1 else parts[0])

    # -- step 3: Hessians without the penalty, and their diagonal sum
    def hessian(self) -> float:
        if self.hess_ctx is None:
            return 0.0
        self.hess_ctx.hessian(egh.EGH_MU_ABS, 0.0)
        return self.hess_ctx.diag_sum()

    # -- step 4: the penalty from the sum over ranks, then the factorisation
    def factor(self, diag_total: float, mu_alpha: float) -> float:
        self.mu = mu_alpha * diag_total / (self.nf * self.nrec)
        if self.hess_ctx is not None:
            self.hess_ctx.set_mu(self.mu)
            self.hess_ctx.factor()
        return self.mu

    # -- step 5: this rank's frequencies' share of the multipliers (zeros without frequencies)
    def deblur(self, resid, out):
        if self.hess_ctx is None:
            out.zero_()
        else:
            self.hess_ctx.deblur(resid, out)

    def _buffer(self, nr, nk):
        ctx = self.green_ctx or self.hess_ctx
        return ctx.transform_buffer(nr, nk)

    def close(self):
        for c in (self.green_ctx, self.hess_ctx):
            if c is not None:
                c.close()


def exchange(sends, recvs, rank, group=None):
    """The all-to-all of step 2 as point-to-point transfers (NCCL and gloo both provide them):
    recvs[r] <- rank r's sends[rank]; this rank's own block is copied locally."""
    import torch.distributed as dist

    ops = []
    for q in range(len(sends)):
        if q == rank:
            if recvs[q].numel():
                recvs[q].copy_(sends[q])
            continue
        if sends[q].numel():
            ops.append(dist.P2POp(dist.isend, sends[q], q, group))
        if recvs[q].numel():
            ops.append(dist.P2POp(dist.irecv, recvs[q], q, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()


def update(shard: Shard, vel, resid, mult, mu_alpha: float, group=None) -> float:
    """One sharded update on this rank (every rank calls it): Green solves, exchange, Hessians,
    penalty, factorisation, deblur.  mult receives the full multipliers on every rank.  Returns
    mu."""
    import torch
    import torch.distributed as dist

    sends = shard.green(vel)
    recvs = shard.receive_buffers()
    exchange(sends, recvs, shard.rank, group)
    shard.assemble(recvs)
    d = torch.tensor([shard.hessian()], dtype=torch.float64, device=mult.device)
    dist.all_reduce(d, group=group)
    mu = shard.factor(float(d.item()), mu_alpha)
    shard.deblur(resid, mult)
    dist.all_reduce(mult, group=group)
    return mu


def update_in_process(shards, vel, resid, mult, mu_alpha: float) -> float:
    """The same update with all ranks' shards in one process, one rank after another (the
    exchange and the sums are local copies and additions): the partitioning checked against an
    unsharded update on one device."""
    import torch

    sends = [s.green(vel) for s in shards]
    for q, s in enumerate(shards):
        recvs = s.receive_buffers()
        for r in range(len(shards)):
            if recvs[r].numel():
                recvs[r].copy_(sends[r][q])
        s.assemble(recvs)
    total = sum(s.hessian() for s in shards)
    mu = None
    for s in shards:
        mu = s.factor(total, mu_alpha)
    mult.zero_()
    part = torch.empty_like(mult)
    for s in shards:
        s.deblur(resid, part)
        mult += part
    return mu
