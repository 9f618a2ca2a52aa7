"""The paper's cheaper variants against the FP64 oracle, through the C ABI.

Band-limited, time-decimated Green functions (Section "Randomized receiver inversion" and the
examples, which resample Green functions to the source's Nyquist rate): the wavelet-driven
solves, every decim-th level transformed and divided by the wavelet's spectrum, compared element
by element with the oracle's restatement, and the Hessian built from them.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

GREEN_TOL, HESS_TOL = 1e-4, 1e-4


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


@pytest.mark.parametrize("decim,dft_chunk", [(1, 0), (4, 64), (7, 32)])
def test_bandlimited_green_and_hessian(decim, dft_chunk):
    import torch
    from paper_2512_16642_gb300 import egh

    c = synth.case_small()
    v32 = np.asarray(c.vel_start, np.float32)
    w32 = synth.ricker(250, c.dt, 8.0, t0=0.125).astype(np.float32)
    grid = oracle.Grid(v32.astype(np.float64), c.dz, c.dx, c.nsponge, c.sponge_R)
    go = oracle.green_dtft_bandlimited(grid, c.rec_iz, c.rec_ix, c.freqs, c.dt, c.nt,
                                       w32.astype(np.float64), decim, workers=4)
    Qo = oracle.add_mu(oracle.hessian_gram(go), 1.0)
    with egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz, c.rec_ix,
                     c.freqs, dft_chunk=dft_chunk, precision=egh.EGH_PREC_MIXED) as ctx:
        ctx.green_bandlimited(torch.from_numpy(v32).cuda(), w32, decim)
        gg = ctx.get_green()
        ctx.hessian(egh.EGH_MU_ABS, 1.0)
        Qg = ctx.get_hessian(False)
        # the Dirac path on the same context afterwards is unaffected
        ctx.green(torch.from_numpy(v32).cuda())
        gd = ctx.get_green()
    assert rel(gg, go) <= GREEN_TOL
    assert rel(Qg, Qo) <= HESS_TOL
    gdo = oracle.green_dtft(grid, c.rec_iz[:3], c.rec_ix[:3], c.freqs, c.dt, c.nt, workers=3)
    assert rel(gd[:3], gdo) <= GREEN_TOL


def test_bandlimited_rejects_bad_input():
    import torch
    from paper_2512_16642_gb300 import egh

    c = synth.case_small()
    v = torch.from_numpy(np.asarray(c.vel_start, np.float32)).cuda()
    with egh.Context(c.nz, c.nx, c.dz, c.dx, c.nsponge, c.sponge_R, c.dt, c.nt, c.rec_iz, c.rec_ix,
                     c.freqs) as ctx:
        for w, d in (([1.0], 0), (np.zeros(5), 2), (np.ones(c.nt + 1), 1), ([np.nan, 1.0], 1)):
            with pytest.raises(egh.EghError) as ei:
                ctx.green_bandlimited(v, w, d)
            assert ei.value.status == egh.EGH_EINVAL
