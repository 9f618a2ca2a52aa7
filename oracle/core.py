"""FP64 CPU ORACLE -- test infrastructure only.

Only tests/, the package smoke check and the benchmark's CPU-baseline leg
may import this module; the product path never does, and this module imports
nothing from the product package.  It is a plain, slow, obviously-correct
restatement of what the method computes, each function citing the passage it
follows.  Pins (checks against things other than itself) live in
tests/test_oracle_pins.py.

Conventions (readings of the paper where it is silent or inconsistent):
  * forward time transform  X(w) = sum_n x_n exp(-i w n dt)  (Section
    "Frequency domain inversion" applies a Fourier transform along time);
  * Hessian entry (i, j) at frequency w is  sum_x ghat_i(w, x) conj(ghat_j(w, x))
    -- the Gram of receiver Green functions over the padded grid (Section
    "Direct Hessian-inverse computation", the outer product G^{ij} summed over
    x), the infinite-record Fourier symbol of the blocks of eq. Hij.  The
    paper's literal W-weighted Fourier diagonal (Section "Computation of the
    Fourier diagonals", eq. weightingfunction, Algorithm 2) is computed too,
    on tiny grids, by three routes (r1_*);
  * mu is one scalar for all frequencies (eq. Qmatrix: mu I in time stays mu I
    under a unitary transform);
  * back to time by band-limited synthesis with weights 2 df_k dt.
"""
from __future__ import annotations

import ctypes
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from . import _build

_lib = None


def _load():
    global _lib
    if _lib is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        f = lib.oracle_fd_run
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        f.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                      ctypes.c_int, dp, dp, ctypes.c_int, ip, dp, ctypes.c_int, ip, dp,
                      ctypes.c_int, dp, dp, dp, ctypes.c_int]
        f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return None if a is None else a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


# ----------------------------------------------------------------------------
# Grid (reading: 20-point sponge padded outside the stated physical grid)
# ----------------------------------------------------------------------------
class Grid:
    """Padded computational grid: physical nz x nx plus nsponge points on all four sides.

    Velocity is extended into the pad by edge replication.  Damping
    eta = eta0 (d/L)^2 per axis (summed over axes), d = distance into the
    sponge, L = nsponge * spacing, eta0 = 1.5 vmax ln(1/R) / L.
    """

    def __init__(self, vel, dz, dx, nsponge, R=1e-3):
        vel = np.asarray(vel, dtype=np.float64)
        self.nz, self.nx = vel.shape
        self.dz, self.dx, self.ns = float(dz), float(dx), int(nsponge)
        ns = self.ns
        self.NZ, self.NX = self.nz + 2 * ns, self.nx + 2 * ns
        self.vel = np.pad(vel, ns, mode="edge")
        vmax = float(vel.max())
        eta = np.zeros((self.NZ, self.NX))
        if ns > 0:
            def prof(N, h):
                i = np.arange(N, dtype=np.float64)
                d = np.maximum(np.maximum(ns - i, i - (N - 1 - ns)), 0.0) * h
                L = ns * h
                return 1.5 * vmax * np.log(1.0 / R) / L * (d / L) ** 2
            eta += prof(self.NZ, self.dz)[:, None]
            eta += prof(self.NX, self.dx)[None, :]
        self.eta = eta

    @property
    def npts(self):
        return self.NZ * self.NX

    def index(self, iz, ix):
        """Flat padded-grid index of physical grid points (iz, ix)."""
        return ((np.asarray(iz) + self.ns) * self.NX + (np.asarray(ix) + self.ns)).astype(np.int32)


def fd_run(grid: Grid, dt, nt, src_p=None, src_f=None, rec_p=None, freqs=None,
           want_snaps=False, nthreads=1):
    """One time-stepping run (C stepper, eq. wave_eq as discretised in fd_oracle.c).

    Returns dict with 'traces' [nrec, nt], 'ghat' [nf, NZ, NX] complex, 'snaps' [nt, NZ, NX]."""
    lib = _load()
    src_p = np.ascontiguousarray(src_p if src_p is not None else np.zeros(0), dtype=np.int32)
    nsrc = src_p.size
    src_f = np.ascontiguousarray(src_f if src_f is not None else np.zeros((0, nt)), dtype=np.float64)
    assert src_f.shape == (nsrc, nt)
    rec_p = np.ascontiguousarray(rec_p if rec_p is not None else np.zeros(0), dtype=np.int32)
    nrec = rec_p.size
    traces = np.zeros((nrec, nt)) if nrec else None
    freqs = np.ascontiguousarray(freqs if freqs is not None else np.zeros(0), dtype=np.float64)
    nf = freqs.size
    ghat = np.zeros((nf, grid.npts, 2)) if nf else None
    snaps = np.zeros((nt, grid.npts)) if want_snaps else None
    vel = np.ascontiguousarray(grid.vel)
    eta = np.ascontiguousarray(grid.eta)
    rc = lib.oracle_fd_run(grid.NZ, grid.NX, grid.dz, grid.dx, float(dt), int(nt), _dp(vel), _dp(eta),
                           nsrc, _ip(src_p), _dp(src_f), nrec, _ip(rec_p), _dp(traces),
                           nf, _dp(freqs), _dp(ghat), _dp(snaps), int(nthreads))
    if rc != 0:
        raise RuntimeError(f"oracle_fd_run failed with {rc}")
    out = {}
    if nrec:
        out["traces"] = traces
    if nf:
        out["ghat"] = (ghat[..., 0] + 1j * ghat[..., 1]).reshape(nf, grid.NZ, grid.NX)
    if want_snaps:
        out["snaps"] = snaps.reshape(nt, grid.NZ, grid.NX)
    return out


def _parallel(fn, items, workers):
    if workers <= 1 or len(items) <= 1:
        return [fn(i) for i in items]
    with ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


def default_workers():
    return max(1, min(16, os.cpu_count() or 1))


# ----------------------------------------------------------------------------
# Step (a): receiver-side Green functions (Section "Direct Hessian-inverse
# computation": g^j is the wavefield of a Dirac source at receiver j; Algorithm 2
# computes them for all active receivers) with their transform at f_k.
# ----------------------------------------------------------------------------
def impulse(nt):
    """Discrete Dirac in time: source amplitude 1 at step 0 (reading of the Dirac source)."""
    f = np.zeros((1, nt))
    f[0, 0] = 1.0
    return f


def green_dtft(grid: Grid, rec_iz, rec_ix, freqs, dt, nt, workers=None, threads_per_run=1):
    """ghat[r, k, z, x] = sum_{n<nt} g^r(n, x) exp(-i 2 pi f_k n dt) over the padded grid."""
    rp = grid.index(rec_iz, rec_ix)
    workers = default_workers() if workers is None else workers

    def one(r):
        return fd_run(grid, dt, nt, src_p=rp[r:r + 1], src_f=impulse(nt), freqs=freqs,
                      nthreads=threads_per_run)["ghat"]

    return np.stack(_parallel(one, list(range(rp.size)), workers))


def green_dtft_bandlimited(grid: Grid, rec_iz, rec_ix, freqs, dt, nt, wavelet, decim, workers=1):
    """Green transforms from a band-limited source, resampled in time (Section "Randomized
    receiver inversion" resamples Green functions to the source's Nyquist rate; the examples use a
    band-pass Ricker source): the solve of receiver r injects wavelet sample s_n at step n (the
    Dirac's convention, sample 0 into level 1), every decim-th level is kept and the transform is
    divided by the wavelet's spectrum,
        ghat[r, k] = decim / S(f_k) * sum_{m: m decim < nt} u^r(m decim) exp(-i 2 pi f_k m decim dt),
        S(f) = sum_n s_n exp(-i 2 pi f n dt)."""
    s = np.asarray(wavelet, dtype=np.float64)
    assert 1 <= s.size <= nt and decim >= 1
    src = np.zeros((1, nt))
    src[0, :s.size] = s
    S = s @ twiddle(freqs, dt, s.size)  # [nf]
    ntd = (nt + decim - 1) // decim
    E = twiddle(freqs, dt * decim, ntd)  # [ntd, nf]
    rp = grid.index(rec_iz, rec_ix)

    def one(r):
        u = fd_run(grid, dt, nt, src_p=rp[r:r + 1], src_f=src, want_snaps=True)["snaps"]
        return np.einsum("mzx,mk->kzx", u[::decim], E) * (decim / S)[:, None, None]

    return np.stack(_parallel(one, list(range(rp.size)), workers))


def green_time(grid: Grid, rec_iz, rec_ix, dt, nt):
    """g[r, n, z, x]: full Green-function time histories (tiny grids only)."""
    rp = grid.index(rec_iz, rec_ix)
    return np.stack([fd_run(grid, dt, nt, src_p=rp[r:r + 1], src_f=impulse(nt), want_snaps=True)["snaps"]
                     for r in range(rp.size)])


# ----------------------------------------------------------------------------
# Step (b): per-frequency Hessian, Gram + mu I (eqs. Qmatrix; Section "Direct
# Hessian-inverse computation": G^{ij} = sum_x g^i g^j^T; Algorithm 2 fills
# (i, j) and conj into (j, i)).
# ----------------------------------------------------------------------------
def hessian_gram(gh):
    """H[k, i, j] = sum_x gh[i, k, x] conj(gh[j, k, x])."""
    nr, nf = gh.shape[:2]
    A = gh.reshape(nr, nf, -1)
    H = np.empty((nf, nr, nr), dtype=np.complex128)
    iu = np.triu_indices(nr, 1)
    for k in range(nf):
        Ak = A[:, k, :]
        Hk = Ak @ Ak.conj().T
        # Algorithm 2: entries (i, j >= i) computed, conj(i, j) placed at (j, i)
        Hk[np.arange(nr), np.arange(nr)] = np.sum(np.abs(Ak) ** 2, axis=1)
        Hk[(iu[1], iu[0])] = Hk[iu].conj()
        H[k] = Hk
    return H


def mu_mean_diag(H, alpha):
    """mu = alpha x mean over frequencies and receivers of Re H_k[i, i] (one scalar)."""
    return float(alpha * np.mean(np.real(np.einsum("kii->ki", H))))


def mu_max_eig(H, alpha):
    """mu = alpha x largest eigenvalue over all frequency blocks (Section "Numerical examples":
    a fraction of the maximum eigenvalue of S S^T; the frequency blocks are its spectrum)."""
    return float(alpha * max(np.linalg.eigvalsh(H[k]).max() for k in range(H.shape[0])))


def add_mu(H, mu):
    Q = H.copy()
    idx = np.arange(H.shape[1])
    Q[:, idx, idx] += mu
    return Q


# ----------------------------------------------------------------------------
# Step (c): factorisation (Algorithm 2 inverts each frequency's matrix; here
# the Hermitian positive-definite blocks are factored as Q = L L^H).
# ----------------------------------------------------------------------------
class NotPositiveDefinite(ValueError):
    def __init__(self, k, j):
        super().__init__(f"frequency {k}: pivot {j} not positive")
        self.k, self.j = k, j


def cholesky(Q):
    """Column-by-column Cholesky of each Hermitian block: L L^H = Q, real positive diagonal."""
    nf, n, _ = Q.shape
    L = np.zeros_like(Q, dtype=np.complex128)
    for k in range(nf):
        A = Q[k]
        Lk = L[k]
        for j in range(n):
            d = np.real(A[j, j]) - np.sum(np.abs(Lk[j, :j]) ** 2)
            if not d > 0.0:
                raise NotPositiveDefinite(k, j)
            Lk[j, j] = np.sqrt(d)
            if j + 1 < n:
                Lk[j + 1:, j] = (A[j + 1:, j] - Lk[j + 1:, :j] @ Lk[j, :j].conj()) / Lk[j, j].real
    return L


def chol_solve(L, B):
    """Solve L L^H X = B per frequency block (forward then backward substitution)."""
    nf, n, _ = L.shape
    X = np.empty_like(B, dtype=np.complex128)
    for k in range(nf):
        Lk = L[k]
        Y = np.zeros_like(B[k], dtype=np.complex128)
        for i in range(n):
            Y[i] = (B[k][i] - Lk[i, :i] @ Y[:i]) / Lk[i, i].real
        Xk = np.zeros_like(Y)
        for i in range(n - 1, -1, -1):
            Xk[i] = (Y[i] - Lk[i + 1:, i].conj() @ Xk[i + 1:]) / Lk[i, i].real
        X[k] = Xk
    return X


# ----------------------------------------------------------------------------
# Step (d): deblur (eq. Qsystemfreq and the per-frequency solve) with transforms
# to and from time.
# ----------------------------------------------------------------------------
def twiddle(freqs, dt, n):
    """exp(-i 2 pi f_k t dt) for t < n, phase reduced as 2 pi frac(f_k t dt); shape [n, nf]."""
    ph = np.outer(np.arange(n, dtype=np.float64), np.asarray(freqs, dtype=np.float64)) * dt
    ph -= np.floor(ph)
    return np.exp(-2j * np.pi * ph)


def dtft_traces(resid, freqs, dt):
    """Dh[k, r, s] = sum_t resid[s, r, t] exp(-i 2 pi f_k t dt)."""
    ns, nr, nt = resid.shape
    E = twiddle(freqs, dt, nt)
    return np.einsum("srt,tk->krs", resid, E)


def synth_weights(freqs, dt, nt):
    """Riemann weights 2 df_k dt of the band-limited inverse transform (one-sided spectrum of
    a real signal); df_k = half the distance between neighbours, the full gap at the ends,
    1/(nt dt) for a single frequency."""
    f = np.asarray(freqs, dtype=np.float64)
    if f.size == 1:
        df = np.array([1.0 / (nt * dt)])
    else:
        df = np.empty_like(f)
        df[1:-1] = 0.5 * (f[2:] - f[:-2])
        df[0] = f[1] - f[0]
        df[-1] = f[-1] - f[-2]
    return 2.0 * df * dt


def synth(X, freqs, dt, nt_d, nt_ref=None):
    """out[s, r, t] = sum_k w_k Re(X[k, r, s] exp(+i 2 pi f_k t dt)), t < nt_d."""
    w = synth_weights(freqs, dt, nt_ref if nt_ref is not None else nt_d)
    E = twiddle(freqs, dt, nt_d).conj()
    return np.real(np.einsum("krs,tk,k->srt", X, E, w))


def deblur(L, resid, freqs, dt, nt_ref=None):
    """Multipliers delta d^e = synth(Q(w)^{-1} DTFT(delta d)) for all sources at once."""
    D = dtft_traces(resid, freqs, dt)
    X = chol_solve(L, D)
    return synth(X, freqs, dt, resid.shape[2], nt_ref=nt_ref), X, D


def deblur_diag(Q, resid, freqs, dt, nt_ref=None):
    """Diagonal-Hessian baseline (the introduction's scaled-identity approximation of earlier
    work; the examples also run the multiplier method keeping only the Hessian's diagonal):
    X_k = D_k / diag(Q_k), then the same synthesis."""
    D = dtft_traces(resid, freqs, dt)
    d = np.real(np.einsum("kii->ki", Q))
    X = D / d[:, :, None]
    return synth(X, freqs, dt, resid.shape[2], nt_ref=nt_ref), X, D


# ----------------------------------------------------------------------------
# Randomised receiver subsets (Section "Randomized receiver inversion": the
# receiver axis is divided into subsets and one receiver is drawn at random from
# each at every iteration).
# ----------------------------------------------------------------------------
_M64 = (1 << 64) - 1


def splitmix64(seed, i):
    """Output number i of SplitMix64 (Steele, Lea and Flood, OOPSLA 2014) from state `seed`:
    the state advances by the golden gamma 0x9E3779B97F4A7C15 before each output, which is
    the state passed through two xor-shift-multiply rounds and a final xor-shift."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & _M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
    return z ^ (z >> 31)


def sample_receivers(nrec, nsub, seed, iteration=0):
    """Subset j = receivers floor(j nrec / nsub) .. floor((j+1) nrec / nsub) - 1; the pick is
    lo + floor(x (hi - lo) / 2^64) with x = splitmix64(seed, iteration * nsub + j)."""
    assert 1 <= nsub <= nrec
    out = []
    for j in range(nsub):
        lo, hi = j * nrec // nsub, (j + 1) * nrec // nsub
        x = splitmix64(seed & _M64, iteration * nsub + j)
        out.append(lo + ((x * (hi - lo)) >> 64))
    return np.array(out, dtype=np.int64)


# ----------------------------------------------------------------------------
# Auxiliary: residuals from Ricker-source modelling (Algorithm 1: delta d_s =
# d_s - P A(m_k)^{-1} b_s).
# ----------------------------------------------------------------------------
def forward_traces(grid: Grid, src_iz, src_ix, rec_iz, rec_ix, wavelet, dt, workers=None):
    """traces[s, r, t] for a point source of signature `wavelet` at each source position."""
    sp = grid.index(src_iz, src_ix)
    rp = grid.index(rec_iz, rec_ix)
    nt = wavelet.size
    workers = default_workers() if workers is None else workers

    def one(s):
        return fd_run(grid, dt, nt, src_p=sp[s:s + 1], src_f=wavelet[None, :], rec_p=rp)["traces"]

    return np.stack(_parallel(one, list(range(sp.size)), workers))


# ----------------------------------------------------------------------------
# Brute-force routes on tiny grids
# ----------------------------------------------------------------------------
def toeplitz_lower(v):
    """T(v): lower-triangular Toeplitz matrix with first column v."""
    n = v.size
    T = np.zeros((n, n))
    for m in range(n):
        T[m, :m + 1] = v[m::-1]
    return T


def hessian_time_domain(g):
    """Eq. Hij: Q^{ij} = sum_x T(g^i(:,x)) T(g^j(:,x))^T; blocks in vec(D) order (receiver-major,
    time fastest).  g[r, n, ...] Green histories."""
    nr, nt = g.shape[:2]
    G = g.reshape(nr, nt, -1)
    npts = G.shape[2]
    Ts = np.zeros((nr, npts, nt, nt))
    for r in range(nr):
        for x in range(npts):
            Ts[r, x] = toeplitz_lower(G[r, :, x])
    Q = np.zeros((nr * nt, nr * nt))
    for i in range(nr):
        for j in range(nr):
            Q[i * nt:(i + 1) * nt, j * nt:(j + 1) * nt] = np.einsum("xml,xnl->mn", Ts[i], Ts[j])
    return Q


def weighting(nt):
    """Eq. weightingfunction: W(m, n) = min(Nt - m, Nt - n), m, n = 0..Nt-1."""
    m = np.arange(nt)
    return np.minimum(nt - m[:, None], nt - m[None, :]).astype(np.float64)


def r1_algorithm2(g):
    """Algorithm 2 literally: G^{ij} = sum_x g^i g^j^T, q^{ij}_xi = sum over n - m = xi of
    (W o G^{ij}), then the 2Nt-length transform (1/2Nt) sum_xi q_xi exp(+i 2 pi k xi / 2Nt)
    (Section "Computation of the Fourier diagonals").  Returns R1[k, i, j], k < 2Nt."""
    nr, nt = g.shape[:2]
    G = g.reshape(nr, nt, -1)
    W = weighting(nt)
    N = 2 * nt
    R = np.zeros((N, nr, nr), dtype=np.complex128)
    for i in range(nr):
        for j in range(i, nr):
            Gij = G[i] @ G[j].T
            WG = W * Gij
            q = np.zeros(N)
            for xi in range(-nt + 1, nt):
                q[xi % N] = np.trace(WG, offset=xi)  # elements with n - m = xi
            qh = np.fft.ifft(q)  # (1/N) sum_xi q_xi exp(+i 2 pi k xi / N)
            R[:, i, j] = qh
            R[:, j, i] = qh.conj()
    return R


def r1_fourier_diagonal(Q, nr, nt):
    """Diagonal of F [[Q^{ij}, 0], [0, 0]] F^H with the unitary 2Nt-point forward DFT F."""
    N = 2 * nt
    k = np.arange(N)[:, None]
    F = np.exp(-2j * np.pi * k * np.arange(nt)[None, :] / N) / np.sqrt(N)  # N x nt (padding dropped)
    R = np.zeros((N, nr, nr), dtype=np.complex128)
    for i in range(nr):
        for j in range(nr):
            B = Q[i * nt:(i + 1) * nt, j * nt:(j + 1) * nt]
            R[:, i, j] = np.einsum("km,mn,kn->k", F, B, F.conj())
    return R


def r1_running_gram(g):
    """(1/2Nt) sum_s Gram of running transforms ghat_s = sum_{n<=s} g_n exp(-i w_k n), using
    W(m, n) = #{s : s >= m, s >= n}."""
    nr, nt = g.shape[:2]
    G = g.reshape(nr, nt, -1)
    N = 2 * nt
    k = np.arange(N)
    E = np.exp(-2j * np.pi * np.outer(np.arange(nt), k) / N)  # [n, k]
    run = np.cumsum(G[:, :, None, :] * E[None, :, :, None], axis=1)  # [r, s, k, x]
    R = np.einsum("iskx,jskx->kij", run, run.conj()) / N
    return R


def r2_on_bins(g):
    """Gram of full-record transforms at the 2Nt FFT bins: sum_x ghat_i conj(ghat_j)."""
    nr, nt = g.shape[:2]
    G = g.reshape(nr, nt, -1)
    N = 2 * nt
    E = np.exp(-2j * np.pi * np.outer(np.arange(nt), np.arange(N)) / N)
    gh = np.einsum("rnx,nk->rkx", G, E)
    return np.einsum("ikx,jkx->kij", gh, gh.conj())


# ----------------------------------------------------------------------------
# Forward and adjoint operators S~ and S~^T (matrix-free), for explicit Hessian
# columns and the Krylov solve the paper compares against (CG, 2 PDE solves per
# iteration).
# ----------------------------------------------------------------------------
class PDECounter:
    def __init__(self):
        self.solves = 0


def apply_S(grid: Grid, dt, nt, rec_p, vol, counter=None):
    """Traces at receivers of the field driven by the volume source vol[n, z, x]."""
    if counter is not None:
        counter.solves += 1
    pts = np.arange(grid.npts, dtype=np.int32)
    src_f = np.ascontiguousarray(vol.reshape(nt, -1).T)
    return fd_run(grid, dt, nt, src_p=pts, src_f=src_f, rec_p=rec_p)["traces"]


def apply_St(grid: Grid, dt, nt, rec_p, traces, counter=None):
    """Adjoint: time-reversed propagation of traces injected at the receivers."""
    if counter is not None:
        counter.solves += 1
    rev = np.ascontiguousarray(traces[:, ::-1])
    snaps = fd_run(grid, dt, nt, src_p=rec_p, src_f=rev, want_snaps=True)["snaps"]
    return snaps[::-1].copy()


def data_fit(grid: Grid, dt, nt, src_p, wavelet, rec_p, d_obs, mult):
    """The paper's Hessian accuracy test (Section "Hessian accuracy test"): the multipliers,
    back-propagated as the adjoint source S^T mult, extend the source b; the extended wavefield
    u^e = A^{-1}(b + S^T mult) sampled at the receivers predicts the data,
        P u^e = P A^{-1} b + S S^T mult   (linearity),
    and the relative error is ||d - P u^e||^2 / ||d||^2.  Returns (d - P u^e, relative error)."""
    d_model = fd_run(grid, dt, nt, src_p=src_p, src_f=np.atleast_2d(wavelet), rec_p=rec_p)["traces"]
    pred = d_model + apply_S(grid, dt, nt, rec_p, apply_St(grid, dt, nt, rec_p, mult))
    r = d_obs - pred
    return r, float(np.sum(r * r) / np.sum(d_obs * d_obs))


def cg_time_domain(grid: Grid, dt, nt, rec_p, d, mu, tol=1e-10, maxiter=500, counter=None):
    """CG on (S~ S~^T + mu I) x = d, d[r, t] (one source gather)."""
    def op(x):
        return apply_S(grid, dt, nt, rec_p, apply_St(grid, dt, nt, rec_p, x, counter), counter) + mu * x

    x = np.zeros_like(d)
    r = d - op(x)
    p = r.copy()
    rs = np.sum(r * r)
    bn = np.sqrt(np.sum(d * d))
    it = 0
    for it in range(1, maxiter + 1):
        Ap = op(p)
        alpha = rs / np.sum(p * Ap)
        x += alpha * p
        r -= alpha * Ap
        rs_new = np.sum(r * r)
        if np.sqrt(rs_new) <= tol * bn:
            break
        p = r + (rs_new / rs) * p
        rs = rs_new
    return x, it
