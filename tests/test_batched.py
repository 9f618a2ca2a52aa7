"""Batched form: the Hessians of several survey patches (different receiver counts, one model)
factored together in one persistent launch replayed as a CUDA graph (egh_batch_*), through the
C ABI.  The batched factors equal the per-context factors bit for bit (each matrix is factored
by one block with the same arithmetic per entry, whatever the block size the first call picks),
and match the FP64 oracle's Cholesky factors.  A patch's Green-function buffers can be released
while its Hessians stay resident.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _patch_ctx(c, rix, prec):
    from paper_2512_16642_gb300 import egh

    return egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt,
                       np.zeros(rix.size, np.int32), rix.astype(np.int32), c.freqs, precision=prec)


@pytest.mark.parametrize("prec", [0, 1])
def test_batched_factor_matches_single_and_oracle(prec):
    import torch
    from paper_2512_16642_gb300 import egh

    c = synth.case_tiny(seed=13, nz=18, nx=40, nsponge=5, nrec=4, nt=160)
    c["freqs"] = np.array([10.0, 18.0, 26.0, 34.0, 42.0])
    patches = [np.arange(0, 40, 6), np.arange(1, 40, 3), np.arange(2, 40, 2)]  # 7, 13, 19 receivers
    v = torch.from_numpy(np.float32(c.vel_true)).cuda()
    ctxs = [_patch_ctx(c, p, prec) for p in patches]
    try:
        single = []
        for ctx in ctxs:
            ctx.green(v)
            ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
            ctx.factor()
            single.append(ctx.get_hessian(True))
        for ctx in ctxs[:2]:
            ctx.release_green()
            with pytest.raises(egh.EghError) as ei:
                ctx.hessian()
            assert ei.value.status == egh.EGH_ESTATE
        with egh.Batch(ctxs) as b:
            for _ in range(2):  # first call tunes and captures, second replays the graph
                b.factor()
                for ctx, L1 in zip(ctxs, single):
                    np.testing.assert_array_equal(ctx.get_hessian(True), L1)
        for ctx in ctxs:
            Q = ctx.get_hessian(False).astype(np.complex128)
            Lo = oracle.cholesky(Q)
            L = ctx.get_hessian(True).astype(np.complex128)
            for k in range(c.freqs.size):
                assert rel(L[k], Lo[k]) <= 1e-3, k
        # a released patch computes its Green functions again
        ctxs[0].green(v)
        ctxs[0].hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        assert np.array_equal(ctxs[0].get_hessian(False), ctxs[0].get_hessian(False))
    finally:
        for ctx in ctxs:
            ctx.close()


def test_batched_factor_reports_failing_patch():
    import torch
    from paper_2512_16642_gb300 import egh

    c = synth.case_tiny(seed=5, nz=8, nx=12, nsponge=2, nrec=3, nt=40)
    c1 = synth.case_tiny(seed=5, nz=8, nx=12, nsponge=2, nrec=3, nt=1)  # zero record: Q = mu I
    ctxs = [_patch_ctx(c, c.rec_ix, 0), _patch_ctx(c1, c1.rec_ix, 0)]
    try:
        v = torch.from_numpy(np.float32(c.vel_true)).cuda()
        ctxs[0].green(v)
        ctxs[0].hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
        ctxs[1].green(v)
        ctxs[1].hessian(egh.EGH_MU_ABS, 0.0)
        with egh.Batch(ctxs) as b:
            with pytest.raises(egh.EghError) as ei:
                b.factor()
            assert ei.value.status == egh.EGH_ENOTPD
            assert ei.value.bad_ctx == 1 and ei.value.bad_freq == 0
    finally:
        for ctx in ctxs:
            ctx.close()
