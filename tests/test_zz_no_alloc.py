"""egh_gram_noalloc, the allocation-free Gram entry point, against egh_hessian and FP64.

For callers that cannot call cudaMalloc (device memory already reserved by another allocator,
or a running service loop that forbids allocation), egh_gram_noalloc computes the per-frequency
Gram from caller-owned device buffers with a fixed scratch array inside the library.  This test
compares it, through the C ABI, with the Hessian of the regular entry point (mu = 0) and with an
FP64 Gram of the same transforms computed on the host, within the Hessian tolerance of the
parity tests, on two calls in a row (the second on a smaller problem, so stale scratch from the
first would show), and checks that the second call takes no device memory."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

HESS_TOL = 1e-4


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _planar(gh, npts):
    nr, nf = gh.shape[:2]
    flat = gh.reshape(nr, nf, -1)
    out = np.zeros((nr, nf, 2, npts), np.float32)
    out[:, :, 0, :flat.shape[2]] = flat.real
    out[:, :, 1, :flat.shape[2]] = flat.imag
    return out


def test_gram_noalloc_matches_hessian_two_calls():
    import torch

    from paper_2512_16642_gb300 import egh

    c = synth.case_tiny(seed=13, nz=20, nx=60, nsponge=6, nrec=70, nt=150)
    c["freqs"] = np.array([8.0, 17.5, 30.0, 44.0])
    with egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz, c.rec_ix,
                     c.freqs) as ctx:
        ctx.green(torch.from_numpy(np.float32(c.vel_true)).cuda())
        assert ctx.hessian(egh.EGH_MU_ABS, 0.0) == 0.0
        ref = ctx.get_hessian(False).astype(np.complex128)
        gh = ctx.get_green()
    nr, nf = gh.shape[:2]
    # the same Gram in FP64 on the host, H[k][i][j] = sum_x g_i conj(g_j)
    g64 = gh.reshape(nr, nf, -1).astype(np.complex128)
    ref64 = np.einsum("ikx,jkx->kij", g64, g64.conj())
    npts = (gh[0, 0].size + 15) // 16 * 16
    d_gh = torch.from_numpy(_planar(gh, npts)).cuda()
    sub = 20
    d_sub = d_gh[:sub].contiguous()
    H = torch.full((nf, nr, nr), float("nan"), dtype=torch.complex64, device="cuda")
    H2 = torch.full((nf, sub, sub), float("nan"), dtype=torch.complex64, device="cuda")

    # call 1: all 70 receivers (3 tiles of 32); its first use on this device loads the scratch
    egh.egh_gram_noalloc(d_gh, nr, nf, npts, H)
    torch.cuda.synchronize()
    h = H.cpu().numpy().astype(np.complex128)
    for k in range(nf):
        assert rel(h[k], ref[k]) <= HESS_TOL, k
        assert rel(h[k], ref64[k]) <= HESS_TOL, k

    # call 2: the first 20 receivers only; it must take no device memory
    free0 = torch.cuda.mem_get_info()[0]
    egh.egh_gram_noalloc(d_sub, sub, nf, npts, H2)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    h2 = H2.cpu().numpy().astype(np.complex128)
    for k in range(nf):
        assert rel(h2[k], ref[k][:sub, :sub]) <= HESS_TOL, k
        assert rel(h2[k], ref64[k][:sub, :sub]) <= HESS_TOL, k


def test_gram_noalloc_rejects_what_it_cannot_do():
    import torch

    from paper_2512_16642_gb300 import egh

    lib = egh.load()

    def raw(gh_ptr, nrec, nfreq, npts, h_ptr):  # the C entry point itself, no wrapper checks
        return lib.egh_gram_noalloc(gh_ptr, nrec, nfreq, npts, h_ptr, torch.cuda.current_stream().cuda_stream)

    H = torch.empty((64, 8, 8), dtype=torch.complex64, device="cuda")
    big = torch.empty((16,), device="cuda")
    # 1000 receivers x 64 frequencies exceed the scratch: refused before any launch
    assert raw(big.data_ptr(), 1000, 64, 16, H.data_ptr()) == egh.EGH_EINVAL
    assert "scratch" in lib.egh_last_error(None).decode()
    host = np.zeros((8, 1, 2, 16), np.float32)  # host memory is refused before any launch
    assert raw(host.ctypes.data, 8, 1, 16, H.data_ptr()) == egh.EGH_EINVAL
    assert raw(big.data_ptr(), 1, 1, 10, H.data_ptr()) == egh.EGH_EINVAL  # npts not a multiple of 16
    with pytest.raises(egh.EghError) as ei:  # the same through the binding
        egh.egh_gram_noalloc(host, 8, 1, 16, H)
    assert ei.value.status == egh.EGH_EINVAL
    # buffers smaller than the sizes say are refused by the binding before the call
    small_gh = torch.zeros((2, 1, 2, 16), device="cuda")
    with pytest.raises(ValueError):
        egh.egh_gram_noalloc(small_gh, 4, 1, 16, H)
    gh_ok = torch.zeros((8, 1, 2, 16), device="cuda")
    small_h = torch.empty((1, 4, 4), dtype=torch.complex64, device="cuda")
    with pytest.raises(ValueError):
        egh.egh_gram_noalloc(gh_ok, 8, 1, 16, small_h)
