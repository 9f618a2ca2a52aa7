"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one oracle function to the mathematics or to values the paper
prints: exact discrete reciprocity, the homogeneous-medium closed form, the
paper's own Fourier-diagonal formulas evaluated by independent routes,
explicit Hessian columns from forward and adjoint solves (eq. Hij), textbook
linear algebra, closed-form transforms, the Krylov solve the paper replaces,
and the counts of Tables 1 and 2.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tiny(nt=24, nz=6, nx=8, nsponge=3, nrec=4, dt=1e-3, R=1e-3, seed=7):
    c = synth.case_tiny(seed=seed, nz=nz, nx=nx, nsponge=nsponge, nrec=nrec, nt=nt, dt=dt)
    g = oracle.Grid(c.vel_true, c.dz, c.dx, c.nsponge, R=R)
    return c, g


@pytest.fixture(scope="module")
def tiny():
    c, g = _tiny()
    gt = oracle.green_time(g, c.rec_iz, c.rec_ix, c.dt, c.nt)
    Q = oracle.hessian_time_domain(gt)
    return c, g, gt, Q


# --- step (a): Green functions ------------------------------------------------
def test_reciprocity_exact():
    """g^i(n, x_j) = g^j(n, x_i): the symmetric damped scheme keeps reciprocity exactly."""
    c, g = _tiny(nt=80, nz=10, nx=12, nsponge=4, nrec=5)
    gt = oracle.green_time(g, c.rec_iz, c.rec_ix, c.dt, c.nt)
    rp = g.index(c.rec_iz, c.rec_ix)
    A = gt.reshape(5, c.nt, -1)[:, :, rp]
    assert np.abs(A - A.transpose(2, 1, 0)).max() <= 1e-12 * np.abs(A).max()


def test_homogeneous_closed_form():
    """dt * DTFT(trace) = R(w) (-i/4) H0^(2)(w r / c) for a Ricker source in a constant medium
    (2D Green function of (1/c^2) d_tt - lap with the exp(-i w t) forward transform)."""
    from scipy.special import hankel2

    c0, dx, dt, nt, n, rpts = 2000.0, 10.0, 1e-3, 1200, 161, 20
    g = oracle.Grid(np.full((n, n), c0), dx, dx, 30, R=1e-4)
    s = n // 2
    rw = synth.ricker(nt, dt, 10.0)
    tr = oracle.fd_run(g, dt, nt, src_p=g.index([s], [s]), src_f=rw[None],
                       rec_p=g.index([s, s + rpts], [s + rpts, s]), nthreads=4)["traces"]
    assert np.abs(tr[0] - tr[1]).max() <= 1e-12 * np.abs(tr).max()  # isotropy of the stencil
    r = rpts * dx
    for f, tol in [(6.0, 2e-2), (10.0, 1e-2), (15.0, 1e-2), (4.0, 4e-2), (20.0, 2e-2)]:
        E = np.exp(-2j * np.pi * f * np.arange(nt) * dt)
        num = dt * (tr[0] @ E)
        ref = dt * (rw @ E) * (-0.25j) * hankel2(0, 2 * np.pi * f * r / c0)
        assert abs(num / ref - 1.0) < tol, (f, abs(num / ref - 1.0))


def test_grid_pad_and_sponge_invariants():
    """The padded grid: velocity replicated from the nearest physical point, no damping on the
    physical grid, damping symmetric about it, growing outward, and additive over the two axes
    (a corner carries both profiles)."""
    rng = np.random.default_rng(2)
    nz, nx, ns = 7, 9, 4
    v = 1500.0 + 1000.0 * rng.random((nz, nx))
    g = oracle.Grid(v, 10.0, 12.5, ns, R=1e-3)
    assert (g.NZ, g.NX) == (nz + 2 * ns, nx + 2 * ns)
    iz = np.clip(np.arange(g.NZ) - ns, 0, nz - 1)
    ix = np.clip(np.arange(g.NX) - ns, 0, nx - 1)
    assert np.array_equal(g.vel, v[np.ix_(iz, ix)])
    e = g.eta
    assert np.all(e[ns:ns + nz, ns:ns + nx] == 0.0)
    assert np.allclose(e, e[::-1, :], rtol=1e-14, atol=0) and np.allclose(e, e[:, ::-1], rtol=1e-14, atol=0)
    zc, xc = g.NZ // 2, g.NX // 2
    assert np.all(np.diff(e[:ns + 1, xc]) < 0) and np.all(np.diff(e[zc, :ns + 1]) < 0)
    assert np.allclose(e[:ns, :ns], e[:ns, xc][:, None] + e[zc, :ns][None, :], rtol=1e-14, atol=0)
    assert np.all(e >= 0.0)


def test_sponge_absorbs_energy():
    """With the sponge the field decays; nothing grows over thousands of steps."""
    c, g = _tiny(nt=3000, nz=20, nx=20, nsponge=10, nrec=1, dt=1e-3)
    rp = g.index([10], [10])
    tr = oracle.fd_run(g, c.dt, c.nt, src_p=rp, src_f=oracle.impulse(c.nt), rec_p=rp)["traces"][0]
    early = np.abs(tr[:300]).max()
    assert np.abs(tr[-500:]).max() < 1e-3 * early
    assert np.all(np.isfinite(tr))


def test_on_the_fly_dtft_matches_stored_history():
    """The stepper's running transform equals the transform of the stored time history
    computed with unreduced phases."""
    c, g = _tiny(nt=64)
    rp = g.index(c.rec_iz[:1], c.rec_ix[:1])
    freqs = np.array([3.0, 7.5, 41.0, 123.4])
    out = oracle.fd_run(g, c.dt, c.nt, src_p=rp, src_f=oracle.impulse(c.nt), freqs=freqs, want_snaps=True)
    n = np.arange(c.nt)
    E = np.exp(-2j * np.pi * np.outer(n * c.dt, freqs))
    ref = np.einsum("nzx,nk->kzx", out["snaps"], E)
    assert np.abs(out["ghat"] - ref).max() <= 1e-12 * np.abs(ref).max()


def test_forward_traces_reciprocity_impulse_and_convolution():
    """Residual modelling (Algorithm 1's S b_s, the residuals' source): (i) swapping sources and
    receivers gives the same traces (source-receiver reciprocity of the symmetric scheme, exact);
    (ii) an impulse signature records the Green function of the source position at the
    receivers; (iii) a Ricker trace is the impulse trace convolved with the signature (the
    scheme is linear and time-invariant from rest), which fixes where each wavelet sample
    enters."""
    c, g = _tiny(nt=70, nz=10, nx=14, nsponge=4, nrec=5)
    s_iz, s_ix = np.array([0, 3, 7], np.int32), np.array([2, 9, 5], np.int32)
    r_iz, r_ix = c.rec_iz, c.rec_ix
    w = synth.ricker(c.nt, c.dt, 60.0)
    T = oracle.forward_traces(g, s_iz, s_ix, r_iz, r_ix, w, c.dt, workers=1)
    Tr = oracle.forward_traces(g, r_iz, r_ix, s_iz, s_ix, w, c.dt, workers=1)
    assert T.shape == (3, 5, c.nt)
    assert np.abs(T - Tr.transpose(1, 0, 2)).max() <= 1e-12 * np.abs(T).max()
    Ti = oracle.forward_traces(g, s_iz, s_ix, r_iz, r_ix, oracle.impulse(c.nt)[0], c.dt, workers=1)
    gt = oracle.green_time(g, s_iz, s_ix, c.dt, c.nt)  # [source][n][z][x]
    rz, rx = r_iz + c.nsponge, r_ix + c.nsponge
    assert np.abs(Ti - gt[:, :, rz, rx].transpose(0, 2, 1)).max() <= 1e-14 * np.abs(Ti).max()
    conv = np.zeros_like(T)
    for t in range(c.nt):
        conv[..., t] = Ti[..., :t + 1] @ w[t::-1]
    assert np.abs(T - conv).max() <= 1e-12 * np.abs(T).max()


def test_bandlimited_impulse_is_the_dirac_transform():
    """A one-sample unit wavelet without decimation (S = 1) gives exactly the Dirac transform."""
    c, g = _tiny(nt=40)
    a = oracle.green_dtft(g, c.rec_iz, c.rec_ix, c.freqs, c.dt, c.nt, workers=1)
    b = oracle.green_dtft_bandlimited(g, c.rec_iz, c.rec_ix, c.freqs, c.dt, c.nt, [1.0], 1)
    assert np.abs(a - b).max() <= 1e-14 * np.abs(a).max()


def test_bandlimited_equals_convolved_dirac_histories():
    """Linearity and time invariance of the stepper: the wavelet-driven solve equals the
    wavelet convolved with the Dirac time histories (sample s_n delayed by n steps), here
    decimated by 3 and divided by the wavelet's spectrum computed as a plain sum."""
    c, g = _tiny(nt=45)
    rng = np.random.default_rng(3)
    s = rng.standard_normal(7)
    D = 3
    gt = oracle.green_time(g, c.rec_iz, c.rec_ix, c.dt, c.nt)  # [r, n, z, x]
    u = np.zeros_like(gt)
    for n in range(s.size):
        u[:, n:] += s[n] * gt[:, :c.nt - n]
    t = np.arange(0, c.nt, D) * c.dt
    S = np.array([np.sum(s * np.exp(-2j * np.pi * f * np.arange(s.size) * c.dt)) for f in c.freqs])
    ref = np.stack([np.einsum("rmzx,m->rzx", u[:, ::D], np.exp(-2j * np.pi * f * t)) * D / S[k]
                    for k, f in enumerate(c.freqs)], axis=1)
    got = oracle.green_dtft_bandlimited(g, c.rec_iz, c.rec_ix, c.freqs, c.dt, c.nt, s, D)
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_bandlimited_approximates_dirac_until_aliasing():
    """With a long record (fields absorbed by the sponge) the band-limited, decimated transform
    approaches the Dirac one while the wavelet's band stays below the decimated Nyquist
    frequency 1/(2 D dt), and fails once it does not (Ricker 15 Hz: D = 10 keeps 50 Hz, D = 30
    folds 16.7 Hz onto the band)."""
    c = synth.case_tiny(nz=30, nx=30, nsponge=10, nt=2400)
    g = oracle.Grid(c.vel_true, c.dz, c.dx, c.nsponge, R=1e-3)
    fr = np.array([10.0, 15.0, 20.0])
    gd = oracle.green_dtft(g, c.rec_iz, c.rec_ix, fr, c.dt, c.nt, workers=1)
    w = synth.ricker(150, c.dt, 15.0)
    err = {}
    for D in (1, 10, 30):
        gb = oracle.green_dtft_bandlimited(g, c.rec_iz, c.rec_ix, fr, c.dt, c.nt, w, D)
        err[D] = max(np.linalg.norm(gb[:, k] - gd[:, k]) / np.linalg.norm(gd[:, k]) for k in range(3))
    assert err[1] <= 1e-3 and err[10] <= 1e-3
    assert err[30] >= 0.1


def test_splitmix64_published_outputs():
    """SplitMix64's first outputs as published with its reference implementation (state 0:
    0xe220a8397b1dcdaf, 0x6e789e6aa1b965f4, 0x06c45d188009454f; state 1234567:
    6457827717110365317, 3203168211198807973)."""
    assert [oracle.splitmix64(0, i) for i in range(3)] == [
        0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    assert [oracle.splitmix64(1234567, i) for i in range(2)] == [
        6457827717110365317, 3203168211198807973]


def test_sample_receivers_one_per_subset_and_uniform():
    """One pick inside each contiguous subset, and each position of a subset equally likely
    (chi-square over many iterations)."""
    nrec, nsub = 231, 100
    counts = np.zeros(3)
    for it in range(3000):
        p = oracle.sample_receivers(nrec, nsub, seed=11, iteration=it)
        lo = np.arange(nsub) * nrec // nsub
        hi = (np.arange(nsub) + 1) * nrec // nsub
        assert np.all((p >= lo) & (p < hi))
        counts += np.bincount(p[hi - lo == 3] - lo[hi - lo == 3], minlength=3)
    exp = counts.sum() / 3
    chi2 = float(np.sum((counts - exp) ** 2 / exp))
    assert chi2 < 13.8  # 2 degrees of freedom, p = 0.001
    assert np.array_equal(oracle.sample_receivers(10, 10, 5), np.arange(10))  # nsub = nrec


def test_deblur_diag_exact_for_diagonal_hessian():
    """For a diagonal Hessian the diagonal baseline is the exact solve."""
    rng = np.random.default_rng(2)
    nf, nr, ns, nt = 3, 5, 2, 64
    d = rng.uniform(1.0, 3.0, (nf, nr))
    Q = np.stack([np.diag(d[k]).astype(np.complex128) for k in range(nf)])
    resid = rng.standard_normal((ns, nr, nt))
    freqs = np.array([20.0, 40.0, 60.0])
    a = oracle.deblur_diag(Q, resid, freqs, 1e-3)[0]
    b = oracle.deblur(oracle.cholesky(Q), resid, freqs, 1e-3)[0]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()


def test_trace_dtft_closed_form():
    """sum_{t<N} cos(w0 t dt) exp(-i w t dt) equals its geometric-series closed form."""
    dt, N, f0 = 1e-3, 1000, 5.3
    x = np.cos(2 * np.pi * f0 * np.arange(N) * dt)
    freqs = np.array([3.0, 5.0, 7.0])
    D = oracle.dtft_traces(x[None, None, :], freqs, dt)[:, 0, 0]

    def geo(a):
        return (1 - np.exp(1j * a * N)) / (1 - np.exp(1j * a))

    w0 = 2 * np.pi * f0 * dt
    for k, f in enumerate(freqs):
        w = 2 * np.pi * f * dt
        ref = 0.5 * (geo(w0 - w) + geo(-w0 - w))
        assert abs(D[k] - ref) <= 1e-10 * abs(ref)


# --- step (b): Hessian ---------------------------------------------------------
def test_r1_three_routes_agree(tiny):
    """The paper's Fourier diagonal of the padded blocks (R1) by Algorithm 2 (W-weighted q_xi,
    2Nt transform), by diag(F Q_pad F^H) of the explicit eq. Hij matrix, and by the Gram of
    running transforms (W(m, n) counts the s >= max(m, n))."""
    c, g, gt, Q = tiny
    a = oracle.r1_algorithm2(gt)
    b = oracle.r1_fourier_diagonal(Q, gt.shape[0], c.nt)
    r = oracle.r1_running_gram(gt)
    s = np.abs(a).max()
    assert np.abs(a - b).max() <= 1e-12 * s
    assert np.abs(a - r).max() <= 1e-12 * s


def test_r1_tends_to_half_gram():
    """For Green functions that decay inside the record, R1 -> (Nt/2Nt) x Gram of full-record
    transforms (the Hessian used on the hot path), with error ~ 1/Nt."""
    errs = []
    for nt in (64, 128, 256, 512):
        c, g = _tiny(nt=nt, nsponge=6, nrec=3, dt=2e-3, R=1e-6)
        gt = oracle.green_time(g, c.rec_iz, c.rec_ix, c.dt, nt)
        R1 = oracle.r1_algorithm2(gt)
        R2 = oracle.r2_on_bins(gt)
        errs.append(np.linalg.norm(R1 - R2 / 2) / np.linalg.norm(R1))
    assert all(e2 < 0.6 * e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 0.06


def test_gram_of_running_dtft_equals_bins(tiny):
    """hessian_gram of the stepper's on-the-fly transforms at the FFT bin frequencies equals the
    Gram computed from stored histories."""
    c, g, gt, Q = tiny
    N = 2 * c.nt
    freqs = np.arange(N) / (N * c.dt)
    gh = oracle.green_dtft(g, c.rec_iz, c.rec_ix, freqs, c.dt, c.nt, workers=1)
    H = oracle.hessian_gram(gh)
    R2 = oracle.r2_on_bins(gt)
    assert np.abs(H - R2).max() <= 1e-10 * np.abs(R2).max()


def test_explicit_columns_from_forward_adjoint_solves(tiny):
    """Columns of S S^T from one adjoint (time-reversed) and one forward solve equal eq. Hij's
    sum_x T(g^i) T(g^j)^T built from stored Green functions (uses reciprocity)."""
    c, g, gt, Q = tiny
    nr, nt = gt.shape[:2]
    rp = g.index(c.rec_iz, c.rec_ix)
    for j, n in [(0, 1), (2, 5), (3, nt - 1), (1, nt // 2)]:
        e = np.zeros((nr, nt))
        e[j, n] = 1.0
        col = oracle.apply_S(g, c.dt, nt, rp, oracle.apply_St(g, c.dt, nt, rp, e))
        ref = Q[:, j * nt + n].reshape(nr, nt)
        assert np.abs(col - ref).max() <= 1e-12 * np.abs(ref).max()


def test_adjoint_dot_product(tiny):
    """S^T is the adjoint of S: <S v, d> = <v, S^T d> for random volume sources v and traces d
    (the time-reversed solve is exact because the scheme is symmetric)."""
    c, g, gt, Q = tiny
    nr, nt = gt.shape[:2]
    rp = g.index(c.rec_iz, c.rec_ix)
    rng = np.random.default_rng(21)
    for _ in range(2):
        v = rng.standard_normal((nt, g.NZ, g.NX))
        d = rng.standard_normal((nr, nt))
        lhs = np.sum(oracle.apply_S(g, c.dt, nt, rp, v) * d)
        rhs = np.sum(v * oracle.apply_St(g, c.dt, nt, rp, d))
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), abs(rhs))


def test_hessian_hermitian_positive_definite():
    c, g = _tiny(nt=200, nsponge=4, nrec=5)
    freqs = np.array([10.0, 20.0, 35.0])
    gh = oracle.green_dtft(g, c.rec_iz, c.rec_ix, freqs, c.dt, c.nt, workers=1)
    H = oracle.hessian_gram(gh)
    mu = oracle.mu_mean_diag(H, 1e-2)
    Q = oracle.add_mu(H, mu)
    assert np.abs(Q - Q.conj().transpose(0, 2, 1)).max() == 0.0
    d = np.einsum("kii->ki", Q)
    assert np.all(np.abs(d.imag) == 0.0) and np.all(d.real > 0)
    for k in range(Q.shape[0]):
        assert np.linalg.eigvalsh(Q[k]).min() >= mu * (1 - 1e-10)
    assert mu == pytest.approx(1e-2 * np.mean(np.sum(np.abs(gh) ** 2, axis=(2, 3))), rel=1e-12)
    mx = oracle.mu_max_eig(H, 1e-2)
    assert mx >= mu


def test_mu_max_eig_closed_form():
    """mu = alpha max_k lambda_max(H_k) on blocks with known spectra: H_k = a_k a_k^H + c_k I has
    lambda_max = |a_k|^2 + c_k (the other eigenvalues are c_k)."""
    rng = np.random.default_rng(3)
    nf, n = 4, 6
    a = rng.standard_normal((nf, n)) + 1j * rng.standard_normal((nf, n))
    cst = np.array([0.5, 3.0, 0.1, 1.0])
    H = np.einsum("ki,kj->kij", a, a.conj()) + cst[:, None, None] * np.eye(n)
    lam = np.sum(np.abs(a) ** 2, axis=1) + cst
    assert oracle.mu_max_eig(H, 0.01) == pytest.approx(0.01 * lam.max(), rel=1e-12)
    # the largest block decides, wherever it sits
    assert oracle.mu_max_eig(H[::-1], 1.0) == pytest.approx(lam.max(), rel=1e-12)


def test_fig1_structure():
    """Fig. 1 (Nt = 7, Nr = 5): the time-domain Q is dense 35 x 35; replacing each block by its
    Fourier diagonal and permuting with Pi (vec(D) -> vec(D^T)) gives 5 x 5 diagonal blocks."""
    c, g = _tiny(nt=7, nrec=5, nx=10)
    gt = oracle.green_time(g, c.rec_iz, c.rec_ix, c.dt, 7)
    Q = oracle.hessian_time_domain(gt)
    assert Q.shape == (35, 35) and np.count_nonzero(np.abs(Q) > 0) > 35 * 35 // 2
    R1 = oracle.r1_algorithm2(gt)  # [2Nt, Nr, Nr]
    N = R1.shape[0]
    Qh = np.zeros((5 * N, 5 * N), dtype=complex)  # receiver-major: each (i, j) block diagonal
    for i in range(5):
        for j in range(5):
            Qh[i * N:(i + 1) * N, j * N:(j + 1) * N] = np.diag(R1[:, i, j])
    perm = np.array([i * N + k for k in range(N) for i in range(5)])
    P = Qh[np.ix_(perm, perm)]
    mask = np.kron(np.eye(N), np.ones((5, 5))) > 0
    assert np.all(P[~mask] == 0)
    for k in range(N):
        assert np.allclose(P[5 * k:5 * k + 5, 5 * k:5 * k + 5], R1[k])


# --- step (c): factorisation ---------------------------------------------------
def _hpd(rng, nf, n, mu=1.0):
    A = rng.standard_normal((nf, n, 3 * n)) + 1j * rng.standard_normal((nf, n, 3 * n))
    return A @ A.conj().transpose(0, 2, 1) + mu * np.eye(n)


def test_cholesky_textbook():
    rng = np.random.default_rng(3)
    Q = _hpd(rng, 3, 17)
    L = oracle.cholesky(Q)
    for k in range(3):
        ref = np.linalg.cholesky(Q[k])
        assert np.abs(L[k] - ref).max() <= 1e-12 * np.abs(ref).max()
        assert np.abs(L[k] @ L[k].conj().T - Q[k]).max() <= 1e-12 * np.abs(Q[k]).max()
        assert np.all(np.triu(L[k], 1) == 0)


def test_cholesky_rejects_indefinite():
    rng = np.random.default_rng(4)
    Q = _hpd(rng, 2, 6)
    Q[1] -= 1e3 * np.eye(6)
    with pytest.raises(oracle.NotPositiveDefinite) as ei:
        oracle.cholesky(Q)
    assert ei.value.k == 1


def test_chol_solve_textbook():
    rng = np.random.default_rng(5)
    Q = _hpd(rng, 2, 9)
    B = rng.standard_normal((2, 9, 4)) + 1j * rng.standard_normal((2, 9, 4))
    X = oracle.chol_solve(oracle.cholesky(Q), B)
    for k in range(2):
        ref = np.linalg.solve(Q[k], B[k])
        assert np.abs(X[k] - ref).max() <= 1e-11 * np.abs(ref).max()


# --- step (d): deblur -----------------------------------------------------------
def test_synthesis_inverts_dense_band():
    """With a dense frequency grid covering a band-limited signal, the band-limited synthesis
    (weights 2 df dt) inverts the forward transform."""
    dt, nt = 1e-3, 800
    s = synth.ricker(nt, dt, 6.0, t0=0.4)
    freqs = np.arange(1, 600) * 0.05  # 0.05 .. 29.95 Hz; Ricker 6 Hz has negligible energy above
    X = oracle.dtft_traces(s[None, None, :], freqs, dt)
    y = oracle.synth(X, freqs, dt, nt)[0, 0]
    assert np.abs(y - s).max() < 2e-3 * np.abs(s).max()


def test_deblur_large_mu_limit():
    """As mu -> inf, Q^{-1} -> I / mu and the deblur reduces to (1/mu) synth(DTFT(d))."""
    rng = np.random.default_rng(6)
    nf, nr, ns, nt, dt = 4, 5, 3, 300, 1e-3
    freqs = np.array([4.0, 5.0, 6.0, 7.0])
    H = _hpd(rng, nf, nr, mu=0.0)
    mu = 1e9
    L = oracle.cholesky(oracle.add_mu(H, mu))
    d = synth.bandlimited_noise(rng, (ns, nr, nt), dt, 3.0, 8.0)
    out, X, D = oracle.deblur(L, d, freqs, dt)
    ref = oracle.synth(D, freqs, dt, nt) / mu
    assert np.abs(out - ref).max() < 1e-6 * np.abs(ref).max()
    # linearity in the residual
    out2, _, _ = oracle.deblur(L, 2.0 * d, freqs, dt)
    assert np.abs(out2 - 2 * out).max() <= 1e-12 * np.abs(out).max()


def test_krylov_agreement():
    """The time-domain Krylov solve the paper replaces: CG on (S S^T + mu I) x = d with two PDE
    solves per iteration matches a dense solve; the direct frequency-domain solution at the
    selected frequencies converges to the transform of that exact solution as the record grows."""
    dt = 2e-3
    errs = []
    for nt in (64, 128, 256, 512):
        c, g = _tiny(nt=nt, nsponge=6, nrec=3, dt=dt, R=1e-6)
        rp = g.index(c.rec_iz, c.rec_ix)
        freqs = np.array([20.0, 30.0, 40.0])
        gh = oracle.green_dtft(g, c.rec_iz, c.rec_ix, freqs, dt, nt, workers=1)
        H = oracle.hessian_gram(gh)
        mu = oracle.mu_mean_diag(H, 1e-2)
        d = np.stack([synth.ricker(nt, dt, 30.0, t0=nt * dt / 2 + 0.01 * r) for r in range(3)])
        cnt = oracle.PDECounter()
        x, it = oracle.cg_time_domain(g, dt, nt, rp, d, mu, tol=1e-12, counter=cnt)
        assert cnt.solves == 2 * it + 2
        if nt == 64:
            gt = oracle.green_time(g, c.rec_iz, c.rec_ix, dt, nt)
            Qt = oracle.hessian_time_domain(gt)
            xd = np.linalg.solve(Qt + mu * np.eye(Qt.shape[0]), d.reshape(-1)).reshape(3, nt)
            assert np.abs(x - xd).max() <= 1e-9 * np.abs(xd).max()
        L = oracle.cholesky(oracle.add_mu(H, mu))
        X = oracle.chol_solve(L, oracle.dtft_traces(d[None], freqs, dt))
        Xt = oracle.dtft_traces(x[None], freqs, dt)
        errs.append(max(np.linalg.norm(X[k] - Xt[k]) / np.linalg.norm(Xt[k]) for k in range(3)))
    assert all(e2 < e1 for e1, e2 in zip(errs, errs[1:])), errs
    assert errs[-1] < 1e-4, errs


def test_data_fit_identity_and_direct_method():
    """The Hessian accuracy test: with the multipliers of the exact time-domain system
    (S S^T + mu I) x = delta d (CG to 1e-12), the data residual of the extended wavefield is
    mu x (d - P u^e = mu delta d^e); the frequency-domain direct method's multipliers (all
    bins up to 120 Hz, 512-step record) fit the data to a small relative error, larger than
    the exact solve's because the Hessian inverse is approximated."""
    dt, nt = 2e-3, 512
    c = synth.case_tiny(nt=nt, nz=6, nx=8, nsponge=6, nrec=3, dt=dt)
    g_true = oracle.Grid(c.vel_true, c.dz, c.dx, c.nsponge, R=1e-6)
    g = oracle.Grid(c.vel_true * 0.97, c.dz, c.dx, c.nsponge, R=1e-6)
    rp = g.index(c.rec_iz, c.rec_ix)
    sp = g.index(np.array([2]), np.array([3]))
    w = synth.ricker(nt, dt, 20.0, t0=0.06)
    d = oracle.fd_run(g_true, dt, nt, src_p=sp, src_f=w[None], rec_p=rp)["traces"]
    dd = d - oracle.fd_run(g, dt, nt, src_p=sp, src_f=w[None], rec_p=rp)["traces"]
    freqs = np.arange(1, int(120 * nt * dt)) / (nt * dt)
    H = oracle.hessian_gram(oracle.green_dtft(g, c.rec_iz, c.rec_ix, freqs, dt, nt, workers=4))
    mu = oracle.mu_mean_diag(H, 1e-2)
    x, _ = oracle.cg_time_domain(g, dt, nt, rp, dd, mu, tol=1e-12)
    r_ex, re_ex = oracle.data_fit(g, dt, nt, sp, w, rp, d, x)
    assert np.linalg.norm(r_ex - mu * x) <= 1e-8 * np.linalg.norm(mu * x)
    m_dir = oracle.deblur(oracle.cholesky(oracle.add_mu(H, mu)), dd[None], freqs, dt)[0][0]
    _, re_dir = oracle.data_fit(g, dt, nt, sp, w, rp, d, m_dir)
    assert re_ex < re_dir < 1e-3


# --- the paper's printed counts -------------------------------------------------
def _rows(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_table1_operation_counts():
    for row in _rows("table1_operation_counts.txt"):
        nz, nx, nr, nt = map(int, row[1:5])
        direct, prop = float(row[5]), float(row[6])
        rz, rx, rr, rt = map(int, row[7:11])
        rand, speed = float(row[11]), float(row[12])
        nxp = nz * nx
        assert nxp * nr ** 2 * nt ** 3 == pytest.approx(direct, rel=5e-3)
        assert nxp * nr ** 2 * nt ** 2 == pytest.approx(prop, rel=5e-3)
        assert rz * rx * rr ** 2 * rt ** 2 == pytest.approx(rand, rel=5e-3)
        assert direct / rand == pytest.approx(speed, rel=3e-2)


def test_table2_pde_solve_counts():
    for row in _rows("table2_pde_solves.txt"):
        ns, cg, gm, cg_s, gm_s, direct = map(int, row[1:])
        assert 2 * cg * ns == cg_s
        assert 2 * gm * ns == gm_s
        assert direct == 100  # one Green-function solve per active receiver (100 receivers)
