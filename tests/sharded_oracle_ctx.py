"""A context with the library's method names backed by the FP64 oracle on the CPU, for testing the
sharded update's partitioning and exchange with gloo ranks (tests only; the product path uses the
library's contexts)."""
import numpy as np
import torch

import oracle


class OracleContext:
    def __init__(self, nz, nx, dz, dx, nsponge, sponge_R, dt, nt, rec_iz, rec_ix, freqs, **kw):
        self.dz, self.dx, self.ns, self.R, self.dt, self.nt = dz, dx, nsponge, sponge_R, dt, nt
        self.NZ, self.NX = nz + 2 * nsponge, nx + 2 * nsponge
        self.rec_iz, self.rec_ix = np.asarray(rec_iz), np.asarray(rec_ix)
        self.freqs = np.asarray(freqs, np.float64)
        self.w = oracle.synth_weights(self.freqs, dt, nt)
        self.gh = self.H = self.Q = self.L = None
        self.mu = 0.0

    def green(self, vel):
        v = np.asarray(vel.numpy() if hasattr(vel, "numpy") else vel, np.float64)
        grid = oracle.Grid(v, self.dz, self.dx, self.ns, self.R)
        self.gh = oracle.green_dtft(grid, self.rec_iz, self.rec_ix, self.freqs, self.dt, self.nt, workers=1)

    def transform_buffer(self, nr, nk):
        return torch.zeros((nr, nk, self.NZ, self.NX), dtype=torch.complex128)

    def export_green(self, k0, nk, out):
        out.copy_(torch.from_numpy(np.ascontiguousarray(self.gh[:, k0:k0 + nk])))

    def import_green(self, t):
        self.gh = t.numpy().copy()

    def hessian(self, mode=None, mu=0.0):
        self.H = oracle.hessian_gram(self.gh)
        self.set_mu(mu)

    def diag_sum(self):
        return float(np.sum(np.einsum("kii->ki", self.Q).real))

    def set_mu(self, mu):
        self.mu = mu
        self.Q = oracle.add_mu(self.H, mu)

    def factor(self):
        self.L = oracle.cholesky(self.Q)

    def set_synthesis_frequencies(self, all_f, k0):
        self.w = oracle.synth_weights(np.asarray(all_f, np.float64), self.dt, self.nt)[k0:k0 + self.freqs.size]

    def deblur(self, resid, out):
        r = resid.numpy().astype(np.float64)
        X = oracle.chol_solve(self.L, oracle.dtft_traces(r, self.freqs, self.dt))
        E = oracle.twiddle(self.freqs, self.dt, r.shape[2]).conj()
        out.copy_(torch.from_numpy(np.real(np.einsum("krs,tk,k->srt", X, E, self.w))))

    def close(self):
        pass
