// Internal declarations of the egh library (not part of the ABI).
//
// Device data layout (all float32 unless stated):
//   wavefield level: [NZ + 2*GUARD][PX], rows z = -GUARD .. NZ+GUARD-1, row pitch PX >= NX + 4
//     (multiple of 64).  Guard rows and columns x >= NX are zero and never written, so the
//     eighth-order stencil reads them as the u = 0 boundary without any bounds test;
//   FD state of a batch of B receivers in pairs: [3][B/2][F] float2, F = (NZ + 2*GUARD) * PX,
//     level n in slot n mod 3 (float2 = receivers 2i, 2i+1 at one point);
//   snapshot ring of the transform: [2 planes hi/lo][2K slots][Bp receivers][G] bf16, level n of
//     a chunk in slot (chunk parity) * K + n mod K, point p = z*PX + x (x >= NX and p >= NZ*PX
//     stay zero); u = hi + lo;
//   Green transforms gh: [nrec][nf][2][G], planes re/im, G = NZ*PX rounded up to 256, point
//     p = z*PX + x (entries with x >= NX or p >= NZ*PX are zero);
//   Hessians Qh, factors Lh: [nf][nrec][nrec] float2 (complex64).
#pragma once
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "egh.h"

#include <complex>
#include <cstdint>
#include <string>
#include <vector>

namespace egh {

constexpr int GUARD = 4;  // stencil radius of the eighth-order Laplacian

// Counts kernel launches (every launch_* wrapper adds its launches); read by egh_get_stats.
void count_launches(int n);
long long launches_so_far();
// Message returned by egh_last_error(NULL) for calls that have no context.
void set_context_free_error(const std::string& msg);

struct Stencil {
  float cx[4];  // c_k / dx^2, k = 1..4
  float cz[4];  // c_k / dz^2
};

struct Layout {
  int nz, nx, ns;  // physical grid and sponge width
  int NZ, NX, PX;  // padded grid and pitch
  long long F;     // floats per wavefield level (with guard rows)
  long long org;   // offset of padded point (0, 0) inside a level: GUARD * PX
  long long G;     // Gram contraction length
};

// ---- egh_api.cu (host helpers shared with the serving loop) -----------------------------------
std::vector<float2> twiddle_table(const std::vector<double>& f, double dt, int len);
std::vector<float> synthesis_weights(const std::vector<double>& f, double dt, int nt);

// ---- fd.cu ------------------------------------------------------------------------------------
// Paired levels: float2 per grid point = (receiver 2i, receiver 2i+1); coef = (c1, c3).
// Snapshot output of one level: hi plane of its slot (receiver 0, point 0) or nullptr for none.
struct SnapOut {
  __nv_bfloat16* lvl;
  long long plane;  // elements from the hi plane to the lo plane
  long long rec;    // elements between receivers (G)
};
cudaError_t launch_check_velocity(const float* vel, long long n, float* d_vmax_bad, cudaStream_t st);
cudaError_t launch_build_coef(const float* vel, const Layout& L, double dz, double dx, double dt,
                              double R, const float* d_vmax, float2* coef, cudaStream_t st);
// tz: rows per warp (12, 16, 18, 20, 24 or 32; 0 = default)
cudaError_t launch_fd_step(const float2* ucur, const float2* uprev, float2* unext,
                           const float2* coef, const Layout& L, const Stencil& S, int npairs,
                           const SnapOut& so, cudaStream_t st, int tz);
int fd_rows_one_wave(const Layout& L, int npairs);
int fd_rows_per_warp_default();
cudaError_t fd_prepare(int nf);  // once per context, before any capture
cudaError_t launch_inject(float2* u, long long pstride, const int* pts, const float2* coef, int nb,
                          float amp, float scale, long long org, const SnapOut& so,
                          cudaStream_t st);
cudaError_t launch_record(const float2* u, long long pstride, const int* rec_pts, int nrec, int nb,
                          float* traces, int nt, int t, cudaStream_t st);
int dft_ncomp(int nf);
size_t dft_smem(int nf);
std::vector<unsigned char> dft_twiddle_tiles(const std::vector<double>& f, double dt, int nt,
                                             const std::vector<std::complex<double>>* scale = nullptr);
cudaError_t make_snap_tmap(CUtensorMap* tm, void* base, long long G, int Bp, int nslot);
// per_sm: CTAs per SM of the persistent transform (1 beside the FD steps, more when it runs
// alone; 0: one CTA per tile); beside_smem: shared memory (reserved parts included) of the FD
// CTAs an SM holds beside the transform (0: none), which sizes the transform's CTAs so that an
// SM holds one of them next to the FD CTAs and never two
cudaError_t launch_dft_tc(const CUtensorMap& tmap, const unsigned char* twt, int nf, int slot0,
                          int kcount, int n0, const Layout& L, float* gh, __nv_bfloat16* ghb,
                          int last, int rec0, int nvalid, int nrec_all, int* err, int expire,
                          int per_sm, long long beside_smem, cudaStream_t st);
// dynamic shared memory of one k_fd_step CTA for npairs receiver pairs
int fd_block_smem(int npairs);
// shared memory (reserved parts included) of the k_fd_step CTAs of npairs pairs and tz rows per
// warp that one SM holds at once; 0 if it cannot be queried
long long fd_sm_smem(int npairs, int tz);

// ---- fd_resident.cu ---------------------------------------------------------------------------
// The padded grid as TR x TC tiles of TZ x TX points (TX % 4 == 0), one block per tile, all
// resident at once; P receiver pairs of a batch held in each block's shared memory.
struct ResGeom {
  int TR, TC, TZ, TX;
  int P;
  size_t smem;  // dynamic shared memory per block
};
// Tile grid with the most pairs (<= want_pairs, <= 8) whose state fits a block's shared memory,
// then the smallest tile; false if not even one pair fits.
bool fd_resident_plan(const Layout& L, int want_pairs, ResGeom* g);
size_t fd_resident_xbuf_float4(const ResGeom& g);  // halo exchange buffer (float4)
size_t fd_resident_flags(const ResGeom& g);        // step counters + abort flag (ints)
int fd_resident_sr_default();                         // rows per z-march segment
bool fd_resident_sr_valid(int sr);                    // 6, 8, 11 or 16
// shared-memory limit of every instance, and a check that the grid is co-resident (sr, np:
// the launch's segment rows and pairs, which set its block size)
cudaError_t fd_resident_prepare(const ResGeom& g, int sr, int np);
// Levels ta .. ta+nsteps-1 of np pairs (ta >= 2), from the state slots of levels ta-1, ta-2 of
// lev ([3][pslot][F]) to the slots of the last two levels; level t's bf16 hi/lo snapshot goes to
// ring slot sbase + (t - t0) / decim when t % decim == 0 (snap: hi plane of ring slot 0, or
// null).  flags: fd_resident_flags(g) ints (zeroed here).  Cooperative launch.
cudaError_t launch_fd_resident(const ResGeom& g, int sr, float2* lev, int pslot, const Layout& L,
                               const float2* coef, const Stencil& S, int np, int ta, int nsteps,
                               int t0, int decim, int sbase, __nv_bfloat16* snap, long long sslot,
                               long long splane, long long srec, float4* xbuf, int* flags,
                               int* err, int expire, cudaStream_t st);

// ---- gram_tc.cu -------------------------------------------------------------------------------
// Gram on the tensor cores from the bf16 hi/lo transforms ghb[nrec][nf][re/im][hi/lo][G].
__host__ __device__ int gram_tc_blocks(int nrec);
size_t gram_tc_workspace_floats(int nrec, int nf, int splits);
int gram_tc_splits(int nrec, int nf, long long G);
cudaError_t make_ghb_tmap(CUtensorMap* tm, void* base, long long G, int nf, int nrec);
cudaError_t launch_gram_tc(const CUtensorMap& tmap, int nrec, int nf, long long G, int splits,
                           float* part, int* err, cudaStream_t st);
cudaError_t launch_gh_to_ghb(const float* gh, int nrec, int nf, long long G, __nv_bfloat16* ghb,
                             cudaStream_t st);
cudaError_t launch_gram_tc_finish(const float* part, int nrec, int nf, int splits, float2* Qh,
                                  cudaStream_t st);

// ---- gram.cu ----------------------------------------------------------------------------------
__host__ __device__ int gram_tiles(int nrec);
size_t gram_workspace_floats(int nrec, int nf, int splits);
cudaError_t launch_gram_partial(const float* gh, int nrec, int nf, long long G, int splits,
                                float* part, cudaStream_t st);
cudaError_t launch_gram_finish(const float* part, int nrec, int nf, int splits, float2* Qh,
                               cudaStream_t st);
cudaError_t launch_diag_sum(const float2* Qh, int nrec, int nf, double* d_sum, cudaStream_t st);
cudaError_t launch_lambda_max(const float2* Qh, int nrec, int nf, double* d_lmax, cudaStream_t st);
cudaError_t launch_add_mu_copy(float2* Qh, float2* Lh, int nrec, int nf, float mu, cudaStream_t st);
cudaError_t launch_add_mu_copy_delta(float2* Qh, float2* Lh, int nrec, int nf, double mu_old,
                                     double mu_new, cudaStream_t st);

// ---- chol.cu ----------------------------------------------------------------------------------
// piv64: FP64 diagonal and pivots (mixed precision)
struct PotrfItem {
  float2* A;    // n x n, factored in place
  int n;
  int* status;  // 0, or the failing pivot + 1
};
size_t potrf_smem(int nmax);
cudaError_t potrf_many_prepare(int nmax);
cudaError_t launch_potrf_many(const PotrfItem* items, int count, int nmax, int blocks, int threads,
                              int piv64, cudaStream_t st);
cudaError_t launch_potrf(float2* Lh, int n, int nf, int* status, cudaStream_t st, int piv64);

// ---- deblur.cu --------------------------------------------------------------------------------
// spectra of ntr = nrec * ns traces into columns s0 .. s0+ns-1 of D[nf][nrec][ld] on the tensor
// cores; twt: the transform's twiddle tiles for at least nt_d levels; err: the flag a bounded
// wait sets (both required; nf <= 64); expire: test hook, the first CTA's first wait runs out
// dev_in: resid is device memory (not a mapping of host memory), which the TMA form needs
cudaError_t launch_trace_dft(const float* resid, int ntr, int nt_d, int nf, int nrec, int ld,
                             int s0, float2* Dh, cudaStream_t st, const unsigned char* twt,
                             int* err, int expire = 0, bool dev_in = false);
cudaError_t launch_trsm(const float2* Lh, int n, int nf, float2* Dh, int ns, cudaStream_t st);
// W = L^{-1} per frequency
cudaError_t launch_trtri(const float2* Lh, int n, int nf, float2* Wh, cudaStream_t st);
// Q^{-1}_k = W_k^H W_k (dense) from the inverse factors
cudaError_t launch_gram_inverse(const float2* Wh, int n, int nf, float2* Ph, cudaStream_t st);
// C_k = A_k B_k (complex, A_k n x n, B_k and C_k n x ld, row-major; C must not alias B) on the
// tensor cores with FP32-class products (three-term bf16 splits), for the nk frequencies of the
// device list kl (all when null); err: the flag a bounded wait sets (solve_tc.cu)
cudaError_t launch_cmm_tc(const float2* A, int n, int nk, const float2* B, int ld, float2* C,
                          const int* kl, int* err, cudaStream_t st);
// diagonal-Hessian baseline: D_k[r][s] /= Q_k[r][r]
cudaError_t launch_diag_solve(const float2* Qh, int n, int nf, float2* Dh, int ns, cudaStream_t st);
// refinement residual R = D - Q X: FP64 arithmetic (fp64) or the compensated FP32 dot product;
// frequencies of the device list kl (nf of them), all when kl is null
cudaError_t launch_resid(const float2* Qh, int n, int nf, const float2* Xh, const float2* Dh,
                         int ns, float2* Rh, bool fp64, cudaStream_t st, const int* kl = nullptr);
inline bool prec_mixed(int prec) { return prec == EGH_PREC_MIXED || prec == EGH_PREC_MIXED_FP64; }
// X_k += R_k (m elements per frequency) for the nk frequencies of kl (all when kl is null)
cudaError_t launch_add_correction(float2* X, const float2* R, long long m, int nk, cudaStream_t st,
                                  const int* kl = nullptr);
// ||Q_k||_F^2 per frequency (FP64 sums) into d_out[nf]
cudaError_t launch_fro2(const float2* Qh, int n, int nf, double* d_out, cudaStream_t st);
// lambda_max(W_k^H W_k) = 1 / lambda_min(Q_k) by power iteration (from below) into lam[nf]
cudaError_t launch_inv_power(const float2* Wh, int n, int nf, double* lam, cudaStream_t st);
// Condition bound of a factorisation from ||Q||_F^2, the power estimate of 1/lambda_min (with a
// margin for its approach from below) and, when known (> 0), mu <= lambda_min.
inline double cond_bound(double fro2, double inv_lmin, double mu) {
  double c = 1.25 * sqrt(fro2) * inv_lmin;
  if (mu > 0 && sqrt(fro2) / mu < c) c = sqrt(fro2) / mu;
  return c;
}
// Frequencies whose solves get one step of iterative refinement: condition bound above this
// threshold.  The products with the inverse factor give solutions with a relative error of about
// 1e-8 cond (measured on the 101x101 case, cond 200-1800) and the bound exceeds cond about
// twofold, so unrefined solutions stay near or below 1e-4, a tenth of the multipliers' tolerance.
constexpr double kRefineCond = 1e4;
// (on the tensor cores when tws, the synthesis twiddle tiles for at least nt_d samples, and err
// are given and 2 nf <= 64; else on the CUDA cores)
// dev_out: mult is device memory (not a mapping of host memory), which the TMA-store form needs;
// scratch: device memory of scratch_bytes for the synthesis operand images (used when at least
// synth_operands_bytes(nf, nrec * ns) and 16-byte aligned; else the kernel gathers them itself)
cudaError_t launch_synth(const float2* Dh, int nrec, int ns, int ld, int s0, int nf, const float* w,
                         const float2* tw, int nt_d, float* mult, cudaStream_t st,
                         const unsigned char* tws = nullptr, int* err = nullptr,
                         bool dev_out = false, unsigned char* scratch = nullptr,
                         size_t scratch_bytes = 0);
size_t synth_operands_bytes(int nf, long long ntr);
std::vector<unsigned char> synth_twiddle_tiles(const std::vector<double>& f, double dt, int nt);

}  // namespace egh
