/*
 * egh.h -- C ABI of the GB300 data-space Hessian library.
 *
 * The library builds, factors and applies the frequency-domain data-space
 * Hessians of multiplier-based extended-source FWI (Sonbolestan & Gholami,
 * arXiv 2512.16642):
 *
 *   Q = S S^T + mu I                                   (eq. Qmatrix)
 *   delta d^e = Q^{-1} delta d, solved per frequency   (eqs. Qsystem, Qsystemfreq)
 *
 * with S = P A(m)^{-1} the forward-modelling operator of the constant-density
 * acoustic wave equation m u_tt - lap u = delta(x - x_s) f(t) (eq. wave_eq).
 * Per model update the pipeline is
 *   egh_green   -> receiver-side Green functions by time-domain finite
 *                  differences, transformed on the fly at the Nf frequencies;
 *   egh_hessian -> Q(w_k) = sum_x ghat_i(w_k, x) conj(ghat_j(w_k, x)) + mu I;
 *   egh_factor  -> Cholesky factors L_k L_k^H = Q(w_k), kept on the device;
 *   egh_deblur  -> residual gathers of many sources to multipliers: forward
 *                  transform in time, two triangular solves per frequency,
 *                  band-limited synthesis back to time.
 *
 * Conventions shared by every call:
 *   - all functions return egh_status; no exception crosses the ABI;
 *   - arrays are C-contiguous, row-major, last index fastest;
 *   - complex values are interleaved (re, im) float pairs ("complex64");
 *   - a pointer documented "host or device" may be either: device memory is
 *     used in place on the given stream; host memory (pageable or pinned) is
 *     copied through an internal staging buffer and the call returns after
 *     its result has reached the host buffer;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); device work is ordered on it and the call may return before
 *     device-only results are complete, except where stated;
 *   - the caller owns every buffer it passes; the context owns the Green
 *     function transforms, the Hessians, their factors, the twiddle tables
 *     and all scratch space until egh_destroy;
 *   - one context is single-threaded; distinct contexts are independent.
 *
 * Time transform convention: X(w) = sum_n x_n exp(-i w n dt).
 */
#ifndef EGH_H
#define EGH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    EGH_OK = 0,
    EGH_EINVAL = 1,   /* bad argument (message in egh_last_error) */
    EGH_ENOMEM = 2,   /* device or host allocation failed */
    EGH_ECUDA = 3,    /* a CUDA runtime call failed */
    EGH_ENOTPD = 4,   /* a Hessian was not positive definite */
    EGH_ESTATE = 5,   /* call out of order (create -> green -> hessian -> factor -> deblur) */
    EGH_ETIMEOUT = 6  /* a bounded device wait ran out */
} egh_status;

typedef enum {
    EGH_MU_ABS = 0,          /* mu = mu_param */
    EGH_MU_REL_MEANDIAG = 1, /* mu = mu_param * mean over k, i of Re H_k[i][i] */
    EGH_MU_REL_MAXEIG = 2    /* mu = mu_param * max over k of lambda_max(H_k)  (Section
                                "Numerical examples": a fraction of the largest eigenvalue of S S^T) */
} egh_mu_mode;

/* Arithmetic of the Hessian, factorisation and solve stages (the transform is bf16x3 on the
 * tensor cores in all three, about 2e-6 relative against FP64):
 *   EGH_PREC_FP32:       Gram as FP32 products and sums on the CUDA cores, FP32 Cholesky,
 *                        triangular substitution (the plain path);
 *   EGH_PREC_MIXED:      Gram as bf16x3 products on the tensor cores with FP32 accumulation (each
 *                        transform stored as bf16 hi + lo; about 1e-5 relative against FP64);
 *                        FP32 Cholesky with FP64 pivots; solves as products with the explicit
 *                        inverse factor; at the frequencies whose condition bound exceeds a
 *                        threshold (egh_set_refinement; default 1e4: unrefined solutions have a
 *                        relative error of about 1e-8 cond, measured, and the bound exceeds cond
 *                        about twofold, so they stay near or below 1e-4) one
 *                        step of iterative refinement follows, whose residual D - Q X is
 *                        accumulated to FP64-class accuracy (about 2^-48 relative) by a
 *                        compensated FP32 dot product;
 *   EGH_PREC_MIXED_FP64: as EGH_PREC_MIXED with the refinement residual accumulated in FP64
 *                        arithmetic (the same rounded residual, several times slower on a GB300,
 *                        whose FP64 rate is a small fraction of its FP32 rate). */
typedef enum {
    EGH_PREC_FP32 = 0,
    EGH_PREC_MIXED = 1,
    EGH_PREC_MIXED_FP64 = 2
} egh_precision;

/*
 * Problem description (Section "Theory"; the discretisation is the library's
 * reading, the paper does not give one):
 *   physical grid nz x nx (z down, x fastest) with spacings dz, dx (m);
 *   an absorbing sponge of nsponge points is padded outside it on all four
 *   sides (damping eta = eta0 (d/L)^2 per axis, eta0 = 1.5 vmax ln(1/R)/L,
 *   R = sponge_R); velocity is extended into the pad by edge replication;
 *   second-order leapfrog in time, eighth-order central differences in space;
 *   Green functions: impulse of unit amplitude at step 0 at each receiver,
 *   injected as 1/(dx dz), nt recorded levels n = 0..nt-1 of step dt (s);
 *   receivers at physical grid points (rec_iz[r], rec_ix[r]);
 *   nfreq (1..64) frequencies freq_hz[k] in (0, 1/(2 dt)), arbitrary (not
 *   tied to an FFT grid).
 * Host arrays are copied by egh_create.
 */
typedef struct {
    int32_t nz, nx;
    double dz, dx;
    int32_t nsponge;
    double sponge_R;
    double dt;
    int32_t nt;
    int32_t nrec;
    const int32_t *rec_iz; /* [nrec], host */
    const int32_t *rec_ix; /* [nrec], host */
    int32_t nfreq;
    const double *freq_hz; /* [nfreq], host */
    int32_t batch_receivers; /* receivers propagated together; 0 = chosen by the library: with
                                the per-step FD kernel and more than 8 receivers, the first
                                egh_green times the FD step per receiver for 8, 16 and 32 (at
                                most nrec) and keeps 16 unless another is 3% faster; else
                                min(nrec, 16) */
    int32_t dft_chunk;       /* levels per transform chunk: 32, 64, ..., 2048; 0 = 512 (the
                                snapshot ring holds 2 chunks x batch_receivers levels); a
                                chunk longer than the record is cut to the smallest power of
                                two, at least 32, that holds nt levels (the same arithmetic in
                                one chunk, a smaller ring) */
    int32_t gram_splits;     /* split of the grid sum in the Gram; 0 = chosen by the library
                                (tensor-core Gram: half, once or twice a default, timed on the
                                first egh_hessian) */
    int32_t fd_rows;         /* FD rows per warp: 12, 16, 18, 20, 24 or 32; 0 = timed on the first
                                egh_green of the context: the smallest count whose tiles fit one
                                wave of resident blocks is kept unless another is 3% faster */
    int32_t precision;       /* egh_precision of the Hessian stage (0 = EGH_PREC_FP32) */
    int32_t fd_kernel;       /* FD solver of the Green stage: 0 or 2 = one kernel per time step,
                                state in global memory (L2-resident), the faster one on a GB300;
                                1 = resident: the batch's wavefield stays in shared memory for a
                                whole transform chunk, one block per SM in a cooperative launch,
                                halos exchanged between neighbouring blocks every step (EGH_EINVAL
                                if it does not fit).  Both give identical levels.  With the
                                resident solver, batch_receivers = 0 takes the most receivers whose
                                state fits (at most 16) and fd_rows does not apply (its rows per
                                segment are timed on the first egh_green) */
    int32_t reserved[2];     /* must be zero */
} egh_config;

typedef struct egh_ctx egh_ctx;

/* Timings (ms, device events) and counters of the last call of each stage. */
typedef struct {
    double green_ms, hessian_ms, factor_ms, deblur_ms;
    int64_t pde_solves;        /* Green-function solves in the last egh_green (= nrec) */
    int64_t point_steps;       /* padded grid points x time steps x receivers of the last egh_green */
    int64_t deblur_sources;    /* sources in the last egh_deblur */
    double mu;                 /* penalty used by the last egh_hessian */
    int32_t nz_pad, nx_pad;    /* padded grid */
    int32_t pitch;             /* row pitch (floats) of the device wavefield layout */
    int32_t batch_receivers, dft_chunk, gram_splits;  /* batch_receivers: in use (the timed
                                                          choice once egh_green has run) */
    int64_t kernel_launches;   /* kernels this library has launched since it was loaded (all contexts) */
    int32_t fd_rows;           /* FD rows per warp in use (0 until chosen) */
    int32_t pad_;
    double fd_ms;              /* last egh_green: device time of the FD steps (per-chunk events) */
    double dft_ms;             /* last egh_green: device time of the transform launches */
    int64_t fd_launches;       /* last egh_green: FD step launches */
    int64_t dft_launches;      /* last egh_green: transform launches */
    double gram_ms;            /* last egh_hessian: device time of the Gram kernel */
    int64_t fd_steps;          /* last egh_green: FD time steps computed (all batches) */
    int32_t fd_kernel;         /* FD solver in use: 1 resident, 2 per step */
    int32_t fd_tiles;          /* resident solver: blocks (tiles) per launch, else 0 */
} egh_stats;

/* Validates the configuration and allocates the device state on the current
 * CUDA device (the Green-stage buffers, the largest, on the first egh_green).
 * Rejects (EGH_EINVAL): non-positive sizes or spacings, a receiver outside the
 * physical grid, a frequency outside (0, 1/(2 dt)), nonzero reserved fields.
 * On failure *out is NULL. */
egh_status egh_create(const egh_config *cfg, egh_ctx **out);

/* Frees everything the context owns.  NULL is a no-op. */
void egh_destroy(egh_ctx *ctx);

/* Step (a): receiver-side Green functions and their transforms (Section
 * "Direct Hessian-inverse computation": one PDE solve per receiver with a
 * Dirac source at the receiver, as Algorithm 2 computes them):
 *   ghat[r][k](x) = sum_{n<nt} g^r(n, x) exp(-i 2 pi f_k n dt)
 * over the whole padded grid.  vel: [nz][nx] float32 velocity (m/s), host or
 * device.  EGH_EINVAL if a velocity is not positive and finite or the CFL
 * number vmax dt sqrt(1/dx^2 + 1/dz^2) exceeds 0.78 (eighth-order leapfrog
 * limit); EGH_ETIMEOUT if a bounded device wait for staged data ran out
 * (the context stays usable).  Blocks until the transforms are complete.
 * Invalidates any previous Hessian and factors. */
egh_status egh_green(egh_ctx *ctx, const float *vel, void *stream);

/* Step (a) in the paper's cheaper form (Section "Randomized receiver inversion" and the
 * examples: Green functions of a band-limited source, resampled in time to the source's Nyquist
 * rate): the same solves with the wavelet s_n (n < nw, host float32) injected at the receiver
 * (sample s_n into level n + 1, the Dirac's level 1 taking s_0), every decim-th level recorded,
 * and the transform divided by the wavelet's spectrum:
 *   ghat[r][k](x) = decim / S(f_k) * sum_{m: m decim < nt} u^r(m decim, x) exp(-i 2 pi f_k m decim dt),
 *   S(f) = sum_{n<nw} s_n exp(-i 2 pi f n dt).
 * Equal to egh_green's result up to the aliasing of the band above 1/(2 decim dt) and the
 * record truncation (the convolved field runs nw steps longer); the transform's work and the
 * snapshot traffic drop by decim.  Inputs and errors as egh_green, plus EGH_EINVAL for nw
 * outside 1 .. nt, decim outside 1 .. nt, a non-finite sample, or |S(f_k)| below 1e-6 of its
 * largest value at some frequency. */
egh_status egh_green_bandlimited(egh_ctx *ctx, const float *vel, const float *wavelet, int32_t nw,
                                 int32_t decim, void *stream);

/* Step (b): per-frequency Hessians Q_k = H_k + mu I (eq. Qmatrix) with
 * H_k[i][j] = sum_x ghat_i conj(ghat_j) (the Gram of G^{ij} = sum_x g^i g^j^T
 * in the frequency domain; (j, i) = conj(i, j) as in Algorithm 2).  mu comes
 * from mode/mu_param; mu_out (host, may be NULL) receives it.  Blocks until mu
 * is known on the host.  Requires egh_green. */
egh_status egh_hessian(egh_ctx *ctx, egh_mu_mode mode, double mu_param, double *mu_out, void *stream);

/* Step (c): Cholesky factors L_k L_k^H = Q_k of all frequencies in one launch
 * (Algorithm 2 inverts each frequency's matrix; the factors stand in for
 * the inverses).  Blocks until the
 * status is known.  EGH_ENOTPD if a pivot is not positive; *bad_freq (host,
 * may be NULL) receives the first failing frequency index, else -1.
 * Requires egh_hessian. */
egh_status egh_factor(egh_ctx *ctx, int32_t *bad_freq, void *stream);

/* Step (d): multipliers delta d^e_s = Q^{-1} delta d_s for ns sources
 * (eq. Qsystem solved per frequency, Section "Frequency domain inversion"):
 *   D[k][r][s]  = sum_{t<nt_d} resid[s][r][t] exp(-i 2 pi f_k t dt)
 *   X_k         = L_k^{-H} L_k^{-1} D_k
 *   mult[s][r][t] = sum_k w_k Re(X_k[r][s] exp(+i 2 pi f_k t dt)),  t < nt_d,
 * w_k = 2 df_k dt, df_k = half the distance between neighbouring frequencies
 * (the full gap at the ends; 1/(nt dt) for a single frequency).
 * resid, mult: [ns][nrec][nt_d] float32, host or device (both the same kind);
 * nt_d may differ from the Green record length; ns = 0 does nothing (the
 * pointers may then be NULL).  Requires egh_factor.  With host buffers the call
 * returns when the multipliers are on the host and reports EGH_ETIMEOUT if a
 * bounded device wait of its transforms ran out; with device buffers it returns
 * before the work completes, and such an expiry is reported by the next call
 * that waits for the device (egh_green, egh_hessian, a host-buffer deblur).
 * A source's multipliers do not depend on the other sources of the call, bit
 * for bit.  Device buffers and pageable host buffers (staged through device
 * buffers) give the same bits; page-locked host buffers are read and written
 * in place through their device mapping by transform kernels of their own,
 * whose rounding differs (at the FP32 level of the transforms). */
egh_status egh_deblur(egh_ctx *ctx, const float *resid, int32_t ns, int32_t nt_d, float *mult, void *stream);

/* Threshold of the selective refinement of the mixed precisions (the paper has no counterpart:
 * its precision is not stated).  egh_factor bounds each cond(Q_k) by ||Q_k||_F times the smaller
 * of 1/mu (lambda_min >= mu) and 1.25 times a 40-step power estimate of lambda_max(Q_k^{-1})
 * computed with the inverse factor; the solves of the frequencies whose bound exceeds the
 * threshold get one refinement step.  0 refines every frequency, infinity none.  Applies from the
 * next egh_factor.  EGH_EINVAL if negative or NaN. */
egh_status egh_set_refinement(egh_ctx *ctx, double threshold);

/* The last egh_factor's condition bounds (cond_bound [nfreq], host, may be NULL) and which
 * frequencies are refined (refined [nfreq] 0/1, host, may be NULL).  Mixed precisions only
 * (EGH_EINVAL otherwise); EGH_ESTATE before egh_factor. */
egh_status egh_get_refinement(egh_ctx *ctx, double *cond_bound, int32_t *refined);

/* Same solve, returning the frequency-domain multipliers X[k][r][s]
 * (complex64, [nfreq][nrec][ns]) instead of synthesising them in time.
 * resid host or device; X device only. */
egh_status egh_deblur_freq(egh_ctx *ctx, const float *resid, int32_t ns, int32_t nt_d, void *X, void *stream);

/* The diagonal-Hessian baseline the paper compares against (its introduction: earlier work
 * replaced the Hessian by a scaled identity; its examples also compare against keeping only
 * the Hessian's diagonal): each frequency's system Q_k X_k = D_k solved with Q_k's
 * diagonal only, X_k[r][s] = D_k[r][s] / Q_k[r][r], then synthesised as egh_deblur.  Same
 * buffers and errors as egh_deblur; requires egh_hessian (no factorisation). */
egh_status egh_deblur_diag(egh_ctx *ctx, const float *resid, int32_t ns, int32_t nt_d, float *mult,
                           void *stream);

/* Randomised receiver subsets (Section "Randomized receiver inversion": the receiver axis is
 * split into nsub subsets and one receiver is drawn at random from each at every iteration).
 * Subset j covers indices floor(j nrec / nsub) .. floor((j + 1) nrec / nsub) - 1; out[j] =
 * lo_j + floor(x_j (hi_j - lo_j) / 2^64) with x_j the SplitMix64 output number
 * iteration * nsub + j of `seed` (counter form: x = mix(seed + (i + 1) * 0x9E3779B97F4A7C15)).
 * Host-only (no device work).  out: [nsub] int32, caller-owned.  EGH_EINVAL unless
 * 1 <= nsub <= nrec and out is not NULL. */
egh_status egh_sample_receivers(int32_t nrec, int32_t nsub, uint64_t seed, uint64_t iteration,
                                int32_t *out);

/* Auxiliary (residual generation, Algorithm 1 delta d_s = d_s - S b_s):
 * traces of point sources with signature `wavelet` ([nt] float32, host) at
 * physical points (src_iz[s], src_ix[s]) (host), recorded at the receivers
 * for the Green record length nt: data [nsrc][nrec][nt] float32, host or
 * device.  vel as in egh_green.  Does not change the Hessian state. */
egh_status egh_forward(egh_ctx *ctx, const float *vel, int32_t nsrc, const int32_t *src_iz,
                       const int32_t *src_ix, const float *wavelet, float *data, void *stream);

/* Copies the transforms of receivers r0..r0+nr-1 to host_out
 * ([nr][nfreq][nz+2 nsponge][nx+2 nsponge] complex64).  Blocks. */
egh_status egh_get_green(egh_ctx *ctx, int32_t r0, int32_t nr, void *host_out);

/* Copies Q_k (factored = 0, Hermitian, both triangles) or L_k (factored = 1,
 * upper triangle zero) to host_out ([nfreq][nrec][nrec] complex64).  Blocks. */
egh_status egh_get_hessian(egh_ctx *ctx, int32_t factored, void *host_out);

/* Allocation-free variant of the Hessian Gram.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc -- a process
 * whose device memory is already reserved by another allocator (a framework's
 * caching pool, an arena sized at start-up), or a service loop that forbids
 * device allocation and its implicit synchronisation once running.  It
 * computes, with the kernels of egh_hessian,
 *   H[k][i][j] = sum_{p<npts} (gh[i][k][0][p] + i gh[i][k][1][p])
 *                            (gh[j][k][0][p] - i gh[j][k][1][p])
 * (no mu added), from caller-owned device buffers:
 *   gh  [nrec][nfreq][2][npts] float32 planes (re, im), 16-byte aligned,
 *       npts a positive multiple of 16 (pad with zeros);
 *   H   [nfreq][nrec][nrec] complex64 output, 8-byte aligned.
 * It allocates nothing: its split-sum workspace is a fixed 32 MiB array in
 * device memory defined by the library, which limits nfreq x (number of 32-
 * receiver tile pairs, t (t + 1) / 2 with t = ceil(nrec / 32)) to 2048; larger
 * sizes return EGH_EINVAL with a message in egh_last_error(NULL).  The first
 * call on a device, made while that device is current, looks up the array's
 * device address.  CUDA loads a library's device code lazily by default, so
 * that first lookup is what reserves the 32 MiB on the device (held until the
 * process exits): make the first call at start-up, before another allocator
 * reserves the device's memory, and before any stream capture.  Later calls
 * take no device memory at all.  All calls
 * share the one array and each overwrites what it uses, so calls that overlap
 * on the GPU (different streams, or different host threads) race and must be
 * ordered by the caller.  Work is queued on `stream`; the call returns
 * without waiting. */
egh_status egh_gram_noalloc(const float *gh, int32_t nrec, int32_t nfreq, int64_t npts, void *H,
                            void *stream);

/* ---- Serving (continuous batching of deblur requests) ------------------------------------- *
 * The paper builds each frequency's Hessian once and reuses it for every source (Algorithm 1's
 * loop over sources, Algorithm 2); a server keeps several factored Hessian sets resident and
 * deblurs residual gathers submitted at any time.  A worker thread admits queued requests in
 * arrival order into `slots` CUDA streams while their device buffers fit in an arena of
 * `hbm_budget_bytes` reserved at creation (admission by HBM budget; no device allocation after
 * creation); queued requests for the same set are packed into one batch (at most
 * `max_batch_sources` sources) that shares the per-frequency solve.  Batches in different slots
 * run concurrently; when one finishes, its memory and slot go to the next requests at once.
 * Results are the same whether a request runs alone or in a batch (each source is its own
 * right-hand side).  Host buffers should be pinned (page-locked) for asynchronous copies and
 * must stay valid until the request is waited for. */
typedef struct egh_server egh_server;

typedef struct {
    int64_t hbm_budget_bytes;  /* device arena for request buffers (>= 1 MiB) */
    int32_t slots;             /* batches in flight at once, 1..16 */
    int32_t max_batch_sources; /* sources packed into one batch, >= 1 */
    int32_t precision;         /* egh_precision of the sets' factorisations and solves */
    int32_t reserved[3];       /* must be zero */
} egh_server_config;

typedef struct {
    int64_t submitted, completed, rejected, sources_done, batches;
    int64_t peak_bytes_in_use;  /* arena high-water mark */
    int32_t peak_in_flight;     /* most batches in flight at once */
    int32_t pad_;
    double p50_s, p99_s, mean_s; /* request latency, submission to completion */
    double span_s;              /* first submission to last completion */
} egh_server_stats;

egh_status egh_server_create(const egh_server_config *cfg, egh_server **out);

/* Adds a resident Hessian set: Q_host [nfreq][nrec][nrec] complex64 (Hermitian positive
 * definite, host; nfreq 1..64) at frequencies freq_hz (Hz) of a record with step dt (s); nt_record sets the
 * synthesis weight of a single frequency (1/(nt_record dt)); requests may have up to max_nt
 * samples per trace.  Q is factored on the device (EGH_ENOTPD if a pivot fails).  Blocks. */
egh_status egh_server_add_set(egh_server *sv, int32_t nrec, int32_t nfreq, const double *freq_hz,
                              double dt, int32_t nt_record, int32_t max_nt, const void *Q_host,
                              int32_t *set_id);

/* Queues the deblur of resid [ns][nrec][nt_d] float32 (host) against set `set_id` into
 * mult [ns][nrec][nt_d] float32 (host).  EGH_ENOMEM if the request alone exceeds the budget.
 * Returns at once with *request_id. */
egh_status egh_server_submit(egh_server *sv, int32_t set_id, const float *resid_host, int32_t ns,
                             int32_t nt_d, float *mult_host, int64_t *request_id);

/* Waits (up to timeout_s) for a request; *latency_s (may be NULL) receives its submission-to-
 * completion time.  EGH_ETIMEOUT with the id kept if it has not finished within timeout_s.
 * Otherwise the id is released and the request's own status is returned: EGH_OK; EGH_ETIMEOUT
 * if a bounded device wait ran out in its batch (its multipliers are not valid; the server
 * stays usable); EGH_ECUDA if its batch could not be launched or the server stopped before
 * running it.  egh_server_last_error tells the cases apart. */
egh_status egh_server_wait(egh_server *sv, int64_t request_id, double timeout_s, double *latency_s);

/* Waits (up to timeout_s) until nothing is queued or in flight.  EGH_ETIMEOUT also when a
 * bounded device wait ran out in some batch since the last drain (those requests returned
 * EGH_ETIMEOUT from egh_server_wait; the server stays usable). */
egh_status egh_server_drain(egh_server *sv, double timeout_s);

/* Test hook of the failure path (the paper has no counterpart): the forward transforms of the
 * next `count` batches each have one bounded device wait run out, on an mbarrier that nothing
 * signals, after about 0.2 ms.  The kernel then records its batch's error flag, lets its copies
 * in flight land, frees its tensor memory and returns, exactly as when staged data never arrive;
 * nothing faults or hangs.  Those batches' requests return EGH_ETIMEOUT. */
egh_status egh_server_test_expire_wait(egh_server *sv, int32_t count);

/* hold != 0: admission pauses (requests already in flight finish; new submissions queue);
 * hold == 0: admission resumes, and the queued requests are packed into batches together
 * (queued requests of one set share a solve up to max_batch_sources).  A drain while held
 * times out unless the queue is empty; destroying a held server still finishes its queue. */
egh_status egh_server_hold(egh_server *sv, int32_t hold);

egh_status egh_server_get_stats(egh_server *sv, egh_server_stats *out);
egh_status egh_server_reset_stats(egh_server *sv);

/* Message of the server's last failure (of the last failed egh_server_create when NULL). */
const char *egh_server_last_error(const egh_server *sv);

/* Finishes queued requests, then frees the server. */
void egh_server_destroy(egh_server *sv);

/* Frees the Green-stage buffers (transforms, bf16 transforms, snapshot ring) of a context whose
 * Hessians are built; the next egh_green allocates them again.  Lets several survey patches
 * keep their factored Hessians resident while only one holds its Green functions.  egh_hessian
 * and egh_get_green then return EGH_ESTATE until egh_green runs again.  Blocks. */
egh_status egh_release_green(egh_ctx *ctx);

/* Test hook of the failure path (the paper has no counterpart).  In the next `count` launches
 * of one kind of kernel of this context, the first block has one bounded device wait run out
 * after about 0.2 ms, on a condition that nothing ever satisfies (an mbarrier phase, or a step
 * count no block publishes); the kernel then takes its failure path exactly as when staged data
 * or a neighbour never arrive: it records the context's error flag, lets its copies in flight
 * land, frees its tensor memory and returns, and the resident solver's other blocks see its
 * abort flag and return too.  Nothing faults or hangs.  The call that waits for that work
 * returns EGH_ETIMEOUT and the context stays usable.  kind: 0 = the Green stage's on-the-fly
 * transform, 1 = the resident FD solver, 2 = the deblur's forward transform.  count = 0
 * cancels. */
egh_status egh_test_expire_wait(egh_ctx *ctx, int32_t kind, int32_t count);

/* ---- Sharded update (several GPUs, one process per GPU) --------------------------------------- *
 * The Green solves are independent per receiver and each frequency's Hessian and factorisation
 * are independent of the others (Algorithm 2), so an update shards across GPUs: rank r solves the
 * receivers of its block for all frequencies (a context with those receivers), one all-to-all
 * exchange moves the transforms from receiver blocks to frequency blocks (egh_export_green on the
 * sending side, egh_import_green on a context that holds every receiver and the rank's
 * frequencies), the penalty needs one all-reduce of the ranks' diagonal sums (egh_hessian with
 * EGH_MU_ABS and mu_param 0, egh_diag_sum, the sum over ranks, egh_set_mu), each rank factors its
 * frequencies, and the multipliers are the sum over ranks of each rank's deblur at its frequencies
 * (the synthesis is linear in the frequencies; egh_set_synthesis_frequencies gives each rank the
 * weights of the full frequency list).  The collectives belong to the caller (e.g. NCCL through
 * torch.distributed). */

/* Copies the transforms of frequencies k0 .. k0+nk-1 of every receiver of the context to d_out
 * ([nrec][nk][re/im][G] float32, device, caller-owned; G = the padded grid's points at the device
 * pitch, egh_stats nz_pad x pitch rounded up to 256).  Requires egh_green.  Queued on stream. */
egh_status egh_export_green(egh_ctx *ctx, int32_t k0, int32_t nk, float *d_out, void *stream);

/* Sets the context's transforms from d_in ([nrec][nfreq][re/im][G] float32, device, the layout of
 * egh_export_green) instead of solving: the context then stands as after egh_green (no snapshot
 * ring is allocated).  Its grid must be the one of the contexts that solved.  Blocks. */
egh_status egh_import_green(egh_ctx *ctx, const float *d_in, void *stream);

/* *out = sum over k, i of Re Q_k[i][i] of the context's current Hessians (with the penalty they
 * hold: none after egh_hessian with EGH_MU_ABS and mu_param 0).  Requires egh_hessian.  Blocks. */
egh_status egh_diag_sum(egh_ctx *ctx, double *out);

/* Replaces the penalty of the current Hessians by mu (Q_k = H_k + mu I; from a penalty of 0 the
 * result is the one egh_hessian gives with that mu, bit for bit).  Factors are invalidated.
 * Requires egh_hessian.  Blocks. */
egh_status egh_set_mu(egh_ctx *ctx, double mu, void *stream);

/* The context's frequencies are entries k0 .. k0+nfreq-1 of the full list all_freq_hz[nall]
 * (host): its synthesis weights become those of the full list (the end weights of a frequency
 * block differ from those of the block alone).  EGH_EINVAL if the entries differ. */
egh_status egh_set_synthesis_frequencies(egh_ctx *ctx, const double *all_freq_hz, int32_t nall,
                                         int32_t k0);

/* ---- Checkpoint of a factored Hessian set ------------------------------------------------- *
 * The Hessians of Algorithm 2 depend only on the model and the receivers; a set built once can
 * be stored and reused by later runs without the Green stage.  File layout (little-endian):
 *   bytes 0-7   magic "EGHQSET1";
 *   bytes 8-15  uint64 length H of the header;
 *   H bytes     JSON header: format, version, nrec, nfreq, freq_hz[nfreq], dt, nt, precision, mu,
 *               rec_iz[nrec], rec_ix[nrec] (physical grid), and per array its name, dtype,
 *               shape and byte offset in the payload;
 *   payload     Q [nfreq][nrec][nrec] complex64 (H_k + mu I, as egh_get_hessian with factored =
 *               0 returns it), then L [nfreq][nrec][nrec] complex64 (the factors, as
 *               egh_get_hessian with factored = 1 returns them).
 * Doubles are written with 17 significant digits, so they read back bit for bit. */

/* Writes the context's factored set to `path` (host file, overwritten).  EGH_ESTATE before
 * egh_factor; EGH_EINVAL if the file cannot be written.  Blocks. */
egh_status egh_save(egh_ctx *ctx, const char *path);

/* Reads a set written by egh_save into a context created with the same receivers, frequencies,
 * record (dt, nt) and precision: Q and mu are loaded and factored again (the same kernels, so the
 * factors equal the saved ones on the same library and device), after which the context stands
 * as after egh_factor: egh_deblur, egh_get_hessian and egh_save work without egh_green.
 * EGH_EINVAL if the file cannot be read, is not such a file, is truncated, or does not match the
 * context; EGH_ENOTPD as egh_factor.  Blocks. */
egh_status egh_load(egh_ctx *ctx, const char *path);

/* ---- Batched factorisation --------------------------------------------------------------- *
 * A batch groups contexts (survey patches of one model, any receiver counts, one device, one
 * precision) whose Hessians are factored together: egh_batch_factor factors every frequency of
 * every context in one persistent launch (blocks take matrices b, b + grid, ...), replayed as a
 * CUDA graph together with the Q -> L copies.  On the first call the launch's block size is
 * chosen by timing the candidates on the batch's own matrices.  Contexts must have passed
 * egh_hessian and must outlive the batch.  EGH_ENOTPD names the first failing context and
 * frequency in *bad_ctx, *bad_freq (host, may be NULL; -1 when all succeed).  Blocks until the
 * pivot status is known. */
typedef struct egh_batch egh_batch;
egh_status egh_batch_create(egh_ctx *const *ctxs, int32_t n, egh_batch **out);
egh_status egh_batch_factor(egh_batch *b, int32_t *bad_ctx, int32_t *bad_freq, void *stream);
const char *egh_batch_last_error(const egh_batch *b);
void egh_batch_destroy(egh_batch *b);

/* Fills *out with the last timings and counters.  Blocks on pending events. */
egh_status egh_get_stats(egh_ctx *ctx, egh_stats *out);

/* Message of the last failure on this context (or of the last failed
 * egh_create when ctx is NULL).  Never NULL. */
const char *egh_last_error(const egh_ctx *ctx);

/* Short name of a status code. */
const char *egh_status_string(egh_status s);

/* ABI version: major * 10000 + minor * 100 + patch. */
int32_t egh_version(void);

#ifdef __cplusplus
}
#endif
#endif /* EGH_H */
