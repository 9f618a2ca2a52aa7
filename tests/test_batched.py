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


def test_batched_factor_mixes_panel_and_column_forms():
    """A patch of 850 receivers (beyond the 800 rows whose 32-column panel fits in shared memory:
    the column form) and one of 13 (the blocked panel form) factored in one persistent launch,
    whose shared memory must hold either form: equal to the per-context factors bit for bit and
    to the FP64 oracle's Cholesky of the same Hessians."""
    import torch
    from paper_2512_16642_gb300 import egh

    c = synth.case_tiny(seed=17, nz=6, nx=860, nsponge=3, nrec=4, nt=24)
    c["freqs"] = np.array([15.0, 30.0])
    patches = [np.arange(0, 850), np.arange(5, 860, 66)]  # 850 and 13 receivers
    v = torch.from_numpy(np.float32(c.vel_true)).cuda()
    ctxs = [_patch_ctx(c, p, egh.EGH_PREC_MIXED) for p in patches]
    try:
        single = []
        for ctx in ctxs:
            ctx.green(v)
            ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha)
            ctx.factor()
            single.append(ctx.get_hessian(True))
            ctx.release_green()
        with egh.Batch(ctxs) as b:
            for _ in range(2):
                b.factor()
                for ctx, L1 in zip(ctxs, single):
                    np.testing.assert_array_equal(ctx.get_hessian(True), L1)
        for ctx in ctxs:
            Q = ctx.get_hessian(False).astype(np.complex128)
            Lo = oracle.cholesky(Q)
            L = ctx.get_hessian(True).astype(np.complex128)
            for k in range(c.freqs.size):
                assert rel(L[k], Lo[k]) <= 1e-3, k
                assert rel(L[k] @ L[k].conj().T, Q[k]) <= 1e-5, k
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


def test_salt_patches_full_size_sampled():
    """The batched form at full size, in the launch configuration the benchmark's salt workload
    times: the 1701x351 salt model, nt 6000, 40 frequencies 2-10 Hz, patches of 161/257/341
    receivers in mixed precision with the default batch, chunk and split choices, each patch's
    Green-stage buffers released after its Hessians, the 120 Hessians factored in one persistent
    launch.  Sampled against the FP64 oracle (run on the host cores beside the GPU work):
    transforms of four receivers (two of the first patch, one of each other) at four of the 40
    frequencies, and the Hessian entries among them (entry (i, j) depends only on g^i and g^j).
    Every one of the 120 batched factors equals the per-context factor bit for bit and
    reproduces its Hessian to FP32 backward-error level; mu is alpha times the mean diagonal."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    from paper_2512_16642_gb300 import egh

    c = synth.case_salt_patches()
    v32 = np.float32(c.vel_true)
    kf = np.array([0, 13, 26, 39])  # 2.0, 4.67, 7.33, 10.0 Hz
    picks = [(0, 0), (0, 160), (1, 128), (2, 340)]  # (patch, receiver within the patch)
    rix = np.array([c.patches[p][i] for p, i in picks], np.int32)
    grid = oracle.Grid(v32.astype(np.float64), c.dz, c.dx, c.nsponge, c.sponge_R)
    tpr = max(1, oracle.default_workers() // rix.size)
    ctxs = []
    with ThreadPoolExecutor(max_workers=1) as ex:
        fut = ex.submit(oracle.green_dtft, grid, np.zeros(rix.size, np.int32), rix, c.freqs[kf], c.dt,
                        c.nt, workers=rix.size, threads_per_run=tpr)
        try:
            vt = torch.from_numpy(v32).cuda()
            gh, Q, L1, mu = {}, [], [], []
            for pi, p in enumerate(c.patches):
                ctx = _patch_ctx(c, p, egh.EGH_PREC_MIXED)
                ctxs.append(ctx)
                ctx.green(vt)
                for t, (pp, i) in enumerate(picks):
                    if pp == pi:
                        gh[t] = ctx.get_green(i, 1)[0][kf]
                mu.append(ctx.hessian(egh.EGH_MU_REL_MEANDIAG, c.mu_alpha))
                ctx.factor()
                Q.append(ctx.get_hessian(False).astype(np.complex128))
                L1.append(ctx.get_hessian(True))
                ctx.release_green()
            with egh.Batch(ctxs) as b:
                for _ in range(2):  # first call tunes and captures, second replays the graph
                    b.factor()
                    for ctx, L in zip(ctxs, L1):
                        np.testing.assert_array_equal(ctx.get_hessian(True), L)
            # the deblur at the largest patch's shape (341 receivers, 40 frequencies: the
            # synthesis of 2 nf > 64 components), from the batched factors
            rd = synth.bandlimited_noise(np.random.default_rng(21), (6, 341, 2000), c.dt, 2.0,
                                         10.0).astype(np.float32)
            rt = torch.from_numpy(rd).cuda()
            mt = torch.empty_like(rt)
            ctxs[2].deblur(rt, mt)
            mult = mt.cpu().numpy()
        finally:
            for ctx in ctxs:
                ctx.close()
        o_gh = fut.result()
    tol = 1e-4
    for t in range(len(picks)):
        for j in range(kf.size):
            assert rel(gh[t][j], o_gh[t, j]) <= tol, (picks[t], j)
    H = oracle.hessian_gram(o_gh)  # [4 frequencies][4][4]
    for k in range(kf.size):
        sub = Q[0][kf[k]][np.ix_([0, 160], [0, 160])] - mu[0] * np.eye(2)
        assert rel(sub, H[k][:2, :2]) <= tol, k
        for t in (2, 3):
            p, i = picks[t]
            d = Q[p][kf[k], i, i] - mu[p]
            assert abs(d - H[k][t, t]) <= tol * abs(H[k][t, t]), (picks[t], k)
    for p in range(3):
        assert mu[p] == pytest.approx(c.mu_alpha * np.mean(np.einsum("kii->ki", Q[p]).real - mu[p]),
                                      rel=tol)
        L = L1[p].astype(np.complex128)
        for k in range(c.freqs.size):
            back = np.linalg.norm(L[k] @ L[k].conj().T - Q[p][k]) / np.linalg.norm(Q[p][k])
            assert back <= 1e-5, (p, k, back)
    # steps a5-a7 element by element: the oracle's Cholesky, solve and synthesis on the GPU's own
    # Hessians of that patch (pinned entry by entry above) for sampled sources
    srcs = [0, 3, 5]
    om = oracle.deblur(oracle.cholesky(Q[2]), rd[srcs].astype(np.float64), c.freqs, c.dt,
                       nt_ref=c.nt)[0]
    for i, s in enumerate(srcs):
        assert rel(mult[s], om[i]) <= 1e-3, s
