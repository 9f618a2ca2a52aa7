// Deblurring of residual gathers against the factored Hessians (eq. Qsystem solved per frequency,
// Section "Frequency domain inversion"):
//   D[k][r][s] = sum_t resid[s][r][t] exp(-i w_k t dt)           (k_trace_tma on device buffers,
//                                                                  k_trace_dft_tc otherwise)
//   X_k = L_k^{-H} L_k^{-1} D_k                                   (k_trsm, all sources as RHS)
//   mixed precision: X_k = Q_k^{-1} D_k with Q_k^{-1} = W_k^H W_k, W_k = L_k^{-1} (k_trtri and
//                    k_cgemm once per factorisation; the product on the tensor cores in
//                    solve_tc.cu), then at ill-conditioned frequencies
//                    X_k += Q_k^{-1} (D_k - Q_k X_k)                (k_resid_dot2 or k_resid64)
//   mult[s][r][t] = sum_k w_k Re(X_k[r][s] exp(+i w_k t dt))      (k_synth_operands + k_synth_tma
//                                                                  on device buffers, k_synth_tc
//                                                                  otherwise; k_synth without the
//                                                                  twiddle tiles)
// Traces are indexed q = s * nrec + r (the [ns][nrec][nt] gather layout); the spectra of one call
// occupy columns s0 .. s0 + ns - 1 of a [nf][nrec][ld] array, so that several gathers (of
// different lengths) can share one solve.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <cmath>
#include <vector>

#include <cooperative_groups.h>
#include <cudaTypedefs.h>

#include "egh_internal.cuh"
#include "tc.cuh"

#include <cuda_bf16.h>

namespace egh {

constexpr int NFMAX = 64;

// CTAs per cluster along the time axis of the forward transform
constexpr int TD_S = 4;

// components of the tensor-core transform: 2 nf rounded up to 32
__host__ __device__ inline int tt_ncomp(int nf) { return (2 * nf + 31) / 32 * 32; }

__device__ __forceinline__ void cp_async4(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(tc::smem_u32(dst)), "l"(src),
               "r"(ok ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(tc::smem_u32(dst)), "l"(src),
               "r"(ok ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }

cudaError_t launch_trace_dft_tc(const float* resid, int ntr, int nt_d, const unsigned char* twt,
                                int nf, int nrec, int ld, int s0, float2* Dh, int* err,
                                int expire, cudaStream_t st);

cudaError_t launch_trace_tma(const float* resid, int ntr, int nt_d, const unsigned char* twt,
                             int nf, int nrec, int ld, int s0, float2* Dh, int* err, int expire,
                             cudaStream_t st);
cudaError_t make_f32_tmap(CUtensorMap* tm, const void* base, long long rows, long long cols,
                          int box_cols, int box_rows, bool swizzle);

cudaError_t launch_trace_dft(const float* resid, int ntr, int nt_d, int nf, int nrec, int ld,
                             int s0, float2* Dh, cudaStream_t st, const unsigned char* twt,
                             int* err, int expire, bool dev_in) {
  // N = 2 nf rounded up to 32 is at most 128 for nf <= 64
  if (nf < 1 || nf > NFMAX || !twt || !err) return cudaErrorInvalidValue;
  const bool vec = (nt_d & 3) == 0 && (reinterpret_cast<uintptr_t>(resid) & 15) == 0;
  if (dev_in && vec && tt_ncomp(nf) <= 64 && ntr > 0)
    return launch_trace_tma(resid, ntr, nt_d, twt, nf, nrec, ld, s0, Dh, err, expire, st);
  return launch_trace_dft_tc(resid, ntr, nt_d, twt, nf, nrec, ld, s0, Dh, err, expire, st);
}

// ---------------------------------------------------------------------------------------------
// Forward transform on the tensor cores: D[q][c] = sum_t resid[q][t] W[c][t] with W the twiddle
// tiles of the Green-stage transform (component c = 2k: cos, 2k + 1: -sin; 64 levels per tile,
// bf16 hi/lo, K-major 128-byte swizzle).  128 traces per CTA (MMA M = 128, 8 warps), N = 2 nf
// rounded up to 32 (at most 128), 64 samples per stage.  The traces are read with coalesced 16-byte loads one stage ahead
// into registers, split u = hi + lo into bf16 (about 2^-17 relative) and written by the threads
// into the K-major swizzled A tiles; one thread issues the bf16x3 MMAs (hi hi, hi lo, lo hi).
// The tensor core's FP32 accumulation drifts over long sums, so blocks of TT_J stages alternate
// between two TMEM buffers and the threads drain each finished block into FP32 register totals.
// The time axis is split over a cluster of TD_S CTAs whose totals meet in rank 0 through
// distributed shared memory, in rank order.  Every wait is bounded.
// ---------------------------------------------------------------------------------------------
constexpr int TT_M = 128, TT_K = 64, TT_J = 8;
constexpr unsigned TT_A = TT_M * 128;  // one A plane (hi or lo): 128 rows x 128 bytes

size_t trace_dft_tc_smem(int nf) {
  const size_t N = tt_ncomp(nf);
  // 2 stages x (A hi + A lo + B hi + B lo), 1024-byte alignment slack
  return 1024 + 2 * (2 * (size_t)TT_A + 2 * N * 128);
}

__device__ __forceinline__ void st_shared_v2(unsigned addr, unsigned a, unsigned b) {
  asm volatile("st.shared.v2.u32 [%0], {%1, %2};" ::"r"(addr), "r"(a), "r"(b) : "memory");
}

template <int N, bool VEC>
__global__ void __cluster_dims__(TD_S, 1, 1) __launch_bounds__(256)
    k_trace_dft_tc(const float* __restrict__ resid, int ntr, int nt_d,
                   const unsigned char* __restrict__ twt, int nf, int nrec, int ld, int s0,
                   float2* __restrict__ Dh, int* __restrict__ err, int expire) {
  extern __shared__ __align__(1024) unsigned char tt_dsm[];
  unsigned char* sm = tt_dsm + ((1024 - (tc::smem_u32(tt_dsm) & 1023)) & 1023);
  constexpr unsigned BT = 2u * N * 128u;           // one twiddle tile (hi + lo)
  constexpr unsigned STG = 2u * TT_A + BT;         // one stage
  __shared__ __align__(8) unsigned long long bars[7];  // bfull[2], mdone[2], blk[2], never
  __shared__ unsigned tslot;
  __shared__ int fail;
  namespace cg = cooperative_groups;
  cg::cluster_group cluster = cg::this_cluster();
  const int tid = threadIdx.x, warp = tid >> 5;
  const int rank = (int)cluster.block_rank();
  const int q0 = (blockIdx.x / TD_S) * TT_M;
  const int nst_all = (nt_d + TT_K - 1) / TT_K, per = (nst_all + TD_S - 1) / TD_S;
  const int sbeg = min(nst_all, rank * per), send = min(nst_all, sbeg + per);
  const int nst = send - sbeg;
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto bfull = [&](int i) { return bar0 + 8u * i; };
  auto mdone = [&](int i) { return bar0 + 8u * (2 + i); };
  auto blkd = [&](int i) { return bar0 + 8u * (4 + i); };
  constexpr unsigned NCOL = 2 * N <= 32 ? 32 : (2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : 256));
  if (warp == 0) tc::tmem_alloc(&tslot, NCOL);
  if (tid == 0) {
    for (int i = 0; i < 7; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    fail = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  auto a_hi = [&](int b) { return tc::smem_u32(sm + (size_t)b * STG); };
  auto b_hi = [&](int b) { return tc::smem_u32(sm + (size_t)b * STG + 2 * TT_A); };
  auto issue_b = [&](int s) {  // twiddle tile of stage s (relative to sbeg) into buffer s % 2
    tc::mbar_expect_tx(bfull(s & 1), BT);
    tc::bulk_g2s(b_hi(s & 1), twt + (size_t)(sbeg + s) * BT, BT, bfull(s & 1));
  };
  // this thread's 8 float4 of a stage: element e = i * 256 + tid -> row e / 16, float4 e % 16
  float4 pre[8];
  auto load = [&](int s) {
    const int t0 = (sbeg + s) * TT_K;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = i * 256 + tid, m = e >> 4, c4 = e & 15;
      const int q = q0 + m, t = t0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (q < ntr) {
        const float* src = resid + (long long)q * nt_d + t;
        if (VEC) {
          if (t < nt_d) v = __ldcs(reinterpret_cast<const float4*>(src));  // nt_d % 4 == 0
        } else {
          if (t < nt_d) v.x = __ldcs(src);
          if (t + 1 < nt_d) v.y = __ldcs(src + 1);
          if (t + 2 < nt_d) v.z = __ldcs(src + 2);
          if (t + 3 < nt_d) v.w = __ldcs(src + 3);
        }
      }
      pre[i] = v;
    }
  };
  auto convert = [&](int b) {  // pre -> A hi / lo planes of buffer b, K-major 128-byte swizzle
    const unsigned ah = a_hi(b);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int e = i * 256 + tid, m = e >> 4, c4 = e & 15;
      const float4 v = pre[i];
      const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
      const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
      const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
      const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
      // samples 4 c4 .. 4 c4 + 3 = bytes 8 c4 .. 8 c4 + 7 of row m: chunk c4 / 2, half c4 % 2
      const unsigned off = (unsigned)((m >> 3) * 1024 + (m & 7) * 128 +
                                      ((((c4 >> 1) ^ (m & 7))) << 4) + ((c4 & 1) << 3));
      st_shared_v2(ah + off, *reinterpret_cast<const unsigned*>(&h01),
                   *reinterpret_cast<const unsigned*>(&h23));
      st_shared_v2(ah + TT_A + off, *reinterpret_cast<const unsigned*>(&l01),
                   *reinterpret_cast<const unsigned*>(&l23));
    }
  };
  // warp w drains TMEM lanes 32 (w % 4) .. (rows) and columns (w / 4) N / 2 .. (a half)
  constexpr int NH = N / 2;
  const int qq = warp & 3, hh = warp >> 2, row = qq * 32 + (tid & 31);
  float tot[NH];
#pragma unroll
  for (int c = 0; c < NH; ++c) tot[c] = 0.f;
  bool ok = true;
  auto drain = [&](int blk) {  // add TMEM buffer blk % 2 into the totals (whole warp)
    const bool got = tc::mbar_wait(blkd(blk & 1), (blk >> 1) & 1);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      return;
    }
    tc::tc_fence_after();
    const unsigned base = tmem + ((unsigned)(qq * 32) << 16) + (unsigned)((blk & 1) * N + hh * NH);
#pragma unroll
    for (int c0 = 0; c0 < NH; c0 += 16) {
      float v[16];
      tc::tmem_ld16(base + (unsigned)c0, v);
#pragma unroll
      for (int i = 0; i < 16; ++i) tot[c0 + i] += v[i];
    }
    tc::tc_fence_before();
  };
  int issued_b = 0, waited_b = 0;  // twiddle copies issued / waited for (thread 0)
  if (nst > 0) {
    if (tid == 0) {
      issue_b(0);
      issued_b = 1;
    }
    load(0);
  }
  const unsigned idesc = tc::idesc_bf16(TT_M, N, 0, 0);
  for (int s = 0; s < nst; ++s) {
    const int b = s & 1, blk = s / TT_J;
    // A and B of buffer b were last read by the MMAs of stage s - 2 (block-uniform decision)
    const bool freed = s < 2 || tc::mbar_wait(mdone(b), ((s - 2) >> 1) & 1);
    if (!__syncthreads_and(freed)) {
      ok = false;
      break;
    }
    convert(b);
    if (s + 1 < nst) load(s + 1);  // the next stage's traces in flight during this stage
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      // test hook: the first CTA's first wait runs out (bars[6] never completes a phase)
      if (s == 0 && expire && blockIdx.x == 0 && !tc::mbar_wait_unsignalled(bar0 + 48u)) {
        fail = 1;
      } else if (!tc::mbar_wait(bfull(b), (s >> 1) & 1)) {
        fail = 1;
      } else {
        waited_b = s + 1;
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)((blk & 1) * N);
        const unsigned ah = a_hi(b), al = ah + TT_A, bh = b_hi(b), bl = bh + N * 128;
        const bool first = s % TT_J == 0;
#pragma unroll
        for (int ks = 0; ks < TT_K / 16; ++ks) {
          const unsigned o = 32u * ks;
          const uint64_t dah = tc::sdesc_sw128(ah + o), dal = tc::sdesc_sw128(al + o);
          const uint64_t dbh = tc::sdesc_sw128(bh + o), dbl = tc::sdesc_sw128(bl + o);
          tc::mma_bf16(dt, dah, dbh, idesc, !(first && ks == 0));
          tc::mma_bf16(dt, dah, dbl, idesc, true);
          tc::mma_bf16(dt, dal, dbh, idesc, true);
        }
        tc::mma_commit(mdone(b));
        if (s % TT_J == TT_J - 1 || s == nst - 1) tc::mma_commit(blkd(blk & 1));
        // the next stage's twiddles go to the other buffer once stage s - 1's MMAs are done
        if (s + 1 < nst) {
          if (s >= 1 && !tc::mbar_wait(mdone(b ^ 1), ((s - 1) >> 1) & 1)) {
            fail = 1;
          } else {
            issue_b(s + 1);
            issued_b = s + 2;
          }
        }
      }
    }
    __syncthreads();
    if (fail) {
      ok = false;
      break;
    }
    // a block's buffer is drained during the next block (its MMAs go to the other buffer)
    if (s % TT_J == 0 && blk >= 1) {
      drain(blk - 1);
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
    }
  }
  if (ok && nst > 0) drain((nst - 1) / TT_J);
  // leave no copy or MMA in flight: copies issued but not consumed, and the last MMAs issued
  // (commit order covers the earlier ones); all bounded
  if (nst > 0 && tid == 0) {
    for (int sc = waited_b; sc < issued_b; ++sc) tc::mbar_wait(bfull(sc & 1), (sc >> 1) & 1);
    const int sl = waited_b - 1;
    if (sl >= 0) tc::mbar_wait(mdone(sl & 1), (sl >> 1) & 1);
  }
  const bool okall = __syncthreads_and(ok) && !fail;
  if (!okall && tid == 0) atomicExch(err, 1);
  // totals to shared memory (the stage buffers are free): P[column][row]
  float* P = reinterpret_cast<float*>(sm);
#pragma unroll
  for (int c = 0; c < NH; ++c) P[(hh * NH + c) * TT_M + row] = okall ? tot[c] : 0.f;
  cluster.sync();
  if (rank == 0) {
    for (int r = 1; r < TD_S; ++r) {
      const float* Pr = cluster.map_shared_rank(P, r);
#pragma unroll
      for (int c = 0; c < NH; ++c) tot[c] += Pr[(hh * NH + c) * TT_M + row];
    }
    const int q = q0 + row;
    if (q < ntr) {
      const int sidx = q / nrec, r = q % nrec;
#pragma unroll
      for (int k = 0; k < NH / 2; ++k) {
        const int kk = hh * (NH / 2) + k;  // components 2 kk, 2 kk + 1 of this half
        if (kk < nf)
          Dh[((long long)kk * nrec + r) * ld + s0 + sidx] = make_float2(tot[2 * k], tot[2 * k + 1]);
      }
    }
  }
  cluster.sync();
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, NCOL);
}

// ---------------------------------------------------------------------------------------------
// Forward transform from device memory, persistent and split by warp role.  The time axis of a
// trace tile is cut into H fixed parts (H = 2 from two stages on: stages [0, nst/2) and
// [nst/2, nst)); a unit is one part of one tile, and each CTA (one per SM) takes an even share
// of the units.  Warp 9 (one thread) streams the units' fp32 samples into a ring of TMA stages
// (128 traces x 64 samples as two 128-byte-swizzled boxes of 32 samples; rows past ntr and
// samples past nt_d read as zero), reloading a slot as soon as it has been read; warp 8 (one
// thread) loads the twiddle tiles and issues the bf16x3 MMAs (A hi against the twiddles' hi and
// lo planes as one MMA of twice the width, then A lo against hi), with A read from tensor
// memory; warps 0-7 (thread = trace row, warps 4-7 the second 32 samples) split each stage into
// bf16 hi / lo, store the A tile into TMEM with tcgen05.st and drain the TMEM blocks (TT_J
// stages each, counted from the part's start) into FP32 register totals, which they add into
// the zeroed spectra at the part's end.  With A in TMEM, shared memory holds only the ring and
// the twiddle tiles.  With two parts
// the spectrum is 0 + a + b in either order, the same bits (floating-point addition commutes),
// and the parts depend on the trace length alone: a trace's spectrum does not depend on the
// other traces of the call.  mbarriers carry every hand-off; every wait is bounded and gives up
// early once another role has failed.
// ---------------------------------------------------------------------------------------------
constexpr int TP_EPI = 256;  // threads of warps 0-7
constexpr int TP_A = 2;  // A tiles in TMEM (the converters fill one while the MMAs read another)
constexpr int TP_B = 4;  // twiddle tiles in flight (loaded TP_B - 2 stages ahead)
// fp32 ring stages: what shared memory holds beside the twiddle tiles
__host__ __device__ constexpr int tp_ring(int N) { return N <= 32 ? 6 : 5; }
// The MMA thread waits for the MMAs of stage g - 2 before reusing a twiddle tile; that phase is
// still the latest one of its mbarrier (mdone of A tile (g - 2) % TP_A) only with two or more A
// tiles: with one, stage g - 1's MMAs may already have completed the next phase.
static_assert(TP_A >= 2 && TP_B >= 3, "two A tiles and three twiddle tiles at least");
constexpr unsigned TP_STAGE = TT_M * TT_K * 4;  // one fp32 ring stage

size_t trace_tma_smem(int N) {
  // ring, twiddle tiles (hi + lo), alignment slack
  return 1024 + (size_t)tp_ring(N) * TP_STAGE + TP_B * 2 * (size_t)N * 128;
}

// the stages of unit u (part u % H of tile u / H)
struct TpUnit {
  int tile, sb, nr;
};
__device__ __forceinline__ TpUnit tp_unit(long long u, int H, int nst) {
  const int half = (int)(u % H);
  TpUnit r;
  r.tile = (int)(u / H);
  r.sb = half * nst / H;
  r.nr = (half + 1) * nst / H - r.sb;
  return r;
}

template <int N>
__global__ void __launch_bounds__(TP_EPI + 64, 1)
    k_trace_tma(const __grid_constant__ CUtensorMap tm_in, int ntr, int nt_d,
                const unsigned char* __restrict__ twt, int nf, int nrec, int ld, int s0, int H,
                float2* __restrict__ Dh, int* __restrict__ err, int expire) {
  constexpr int R = tp_ring(N);
  constexpr unsigned BT = 2u * N * 128u;  // one twiddle tile (hi + lo)
  constexpr int NH = N / 2;
  extern __shared__ __align__(1024) unsigned char tp_dsm[];
  unsigned char* sm = tp_dsm + ((1024 - (tc::smem_u32(tp_dsm) & 1023)) & 1023);
  constexpr int NB = TP_B, NA = TP_A;
  // rfull[R], rempty[R], bfull[NB], afull[NA], mdone[NA], blkd[2], tempty[2], never
  __shared__ __align__(8) unsigned long long bars[2 * R + NB + 2 * NA + 5];
  __shared__ unsigned tslot;
  __shared__ int fail_s;
  volatile int* fail = &fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ntile = (ntr + TT_M - 1) / TT_M, nst = (nt_d + TT_K - 1) / TT_K;
  const long long U = (long long)ntile * H;
  const long long u0 = U * blockIdx.x / gridDim.x;
  const int n = (int)(U * (blockIdx.x + 1) / gridDim.x - u0);  // units of this CTA
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto rfull = [&](int i) { return bar0 + 8u * i; };
  auto rempty = [&](int i) { return bar0 + 8u * (R + i); };
  auto bfull = [&](int i) { return bar0 + 8u * (2 * R + i); };
  // A tile g % NA: filled for stage g (afull), read by stage g's MMAs (mdone); phase g / NA
  auto afull = [&](int g) { return bar0 + 8u * (2 * R + NB + g % NA); };
  auto mdone = [&](int g) { return bar0 + 8u * (2 * R + NB + NA + g % NA); };
  auto blkd = [&](int i) { return bar0 + 8u * (2 * R + NB + 2 * NA + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (2 * R + NB + 2 * NA + 2 + i); };
  const unsigned never = bar0 + 8u * (2 * R + NB + 2 * NA + 4);
  // TMEM: two block buffers of 2N columns ([0, N) hi.hi + lo.hi, [N, 2N) hi.lo), then the A tiles
  // at column ACOL: per tile 32 columns of hi (64 samples, two bf16 each) and 32 of lo
  constexpr unsigned ACOL = 4 * N, TCOLS = 4 * N + 64 * TP_A <= 256 ? 256 : 512;
  if (warp == 0) tc::tmem_alloc(&tslot, TCOLS);
  if (tid == 0) {
    for (int i = 0; i < R; ++i) {
      tc::mbar_init(rfull(i), 1);
      tc::mbar_init(rempty(i), TP_EPI);
    }
    for (int i = 0; i < NB; ++i) tc::mbar_init(bfull(i), 1);
    for (int i = 0; i < NA; ++i) {
      tc::mbar_init(afull(i), TP_EPI);
      tc::mbar_init(mdone(i), 1);
    }
    for (int i = 0; i < 2; ++i) {
      tc::mbar_init(blkd(i), 1);
      tc::mbar_init(tempty(i), TP_EPI);
    }
    tc::mbar_init(never, 1);
    fail_s = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  const unsigned ring0 = tc::smem_u32(sm);
  const unsigned bbuf0 = ring0 + R * TP_STAGE;
  // stages of this CTA in order: unit i, stage s of the unit
  struct Cur {
    int i, s;
    TpUnit t;
  };
  auto cur_init = [&](Cur& c) {
    c.i = 0;
    c.s = 0;
    c.t = tp_unit(u0, H, nst);
  };
  auto cur_next = [&](Cur& c) {
    if (++c.s == c.t.nr) {
      c.s = 0;
      if (++c.i < n) c.t = tp_unit(u0 + c.i, H, nst);
    }
  };
  bool ok = true;
  if (warp == 8) {
    if (lane == 0 && n > 0) {
      int G = 0;  // stages of this CTA
      for (int i = 0; i < n; ++i) G += tp_unit(u0 + i, H, nst).nr;
      Cur mc, bc;  // next MMA stage, next twiddle load
      cur_init(mc);
      cur_init(bc);
      auto issue_b = [&](int g) {
        tc::mbar_expect_tx(bfull(g % NB), BT);
        tc::bulk_g2s(bbuf0 + (g % NB) * BT, twt + (size_t)(bc.t.sb + bc.s) * BT, BT, bfull(g % NB));
        cur_next(bc);
      };
      // A hi against the twiddles' hi and lo planes in one MMA (N = 2N: the planes are adjacent
      // rows of one K-major tile), then A lo against the hi plane
      const unsigned idesc2 = tc::idesc_bf16(TT_M, 2 * N, 0, 0), idesc = tc::idesc_bf16(TT_M, N, 0, 0);
      int issued_b = 0, issued_m = 0, b = -1;
      for (; issued_b < min(NB - 1, G); ++issued_b) issue_b(issued_b);
      // test hook: the first CTA's first wait runs out (`never` completes no phase)
      if (expire && blockIdx.x == 0 && !tc::mbar_wait_unsignalled(never)) ok = false;
      for (int g = 0; g < G && ok; ++g) {
        const int s = mc.s;
        const bool first = s % TT_J == 0, last = (s + 1) % TT_J == 0 || s == mc.t.nr - 1;
        if (first) ++b;  // TMEM block of this stage
        // twiddles of stage j = issued_b (at most g + NB - 2) into the buffer that stage j - NB's
        // MMAs read, issued two stages ago (so that this thread does not wait on the MMAs it
        // has just issued)
        while (issued_b < G && issued_b <= g + NB - 2) {
          const int jm = issued_b - NB;
          if (jm >= 0 && !tc::mbar_wait_or(mdone(jm), (jm / NA) & 1, fail)) {
            ok = false;
            break;
          }
          issue_b(issued_b);
          ++issued_b;
        }
        if (!ok) break;
        if (!tc::mbar_wait_or(afull(g), (g / NA) & 1, fail) ||
            !tc::mbar_wait_or(bfull(g % NB), (g / NB) & 1, fail)) {
          ok = false;
          break;
        }
        // a block's TMEM buffer was drained two blocks ago
        if (first && b >= 2 && !tc::mbar_wait_or(tempty(b & 1), ((b - 2) >> 1) & 1, fail)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)((b & 1) * 2 * N);
        const unsigned ah = tmem + ACOL + (unsigned)((g % NA) * 64), al = ah + 32;
        const unsigned bh = bbuf0 + (g % NB) * BT;
#pragma unroll
        for (int ks = 0; ks < TT_K / 16; ++ks) {
          const uint64_t dbh = tc::sdesc_sw128(bh + 32u * ks);
          tc::mma_bf16_ta(dt, ah + 8u * ks, dbh, idesc2, !(first && ks == 0));
          tc::mma_bf16_ta(dt, al + 8u * ks, dbh, idesc, true);
        }
        tc::mma_commit(mdone(g));
        issued_m = g + 1;
        if (last) tc::mma_commit(blkd(b & 1));
        cur_next(mc);
      }
      if (!ok) *fail = 1;
      // leave no copy or MMA in flight: the last issue of each twiddle buffer and the last MMAs
      // (bounded)
      for (int i = 0; i < NB; ++i) {
        const int nis = issued_b > i ? (issued_b - 1 - i) / NB + 1 : 0;
        if (nis > 0) tc::mbar_wait(bfull(i), (nis - 1) & 1);
      }
      if (issued_m > 0) tc::mbar_wait(mdone(issued_m - 1), ((issued_m - 1) / NA) & 1);
    }
  } else if (warp == 9) {
    // the ring: a slot is loaded again as soon as the converters have read it
    if (lane == 0 && n > 0) {
      int G = 0;
      for (int i = 0; i < n; ++i) G += tp_unit(u0 + i, H, nst).nr;
      Cur lc;
      cur_init(lc);
      int issued_r = 0;
      for (; issued_r < G; ++issued_r) {
        const int slot = issued_r % R;
        if (issued_r >= R && !tc::mbar_wait_or(rempty(slot), (issued_r / R - 1) & 1, fail)) {
          ok = false;
          break;
        }
        tc::mbar_expect_tx(rfull(slot), TP_STAGE);
        // two boxes of 128 traces x 32 samples (128-byte rows, 128-byte swizzle)
        for (int h = 0; h < 2; ++h)
          tc::tma_load_2d(ring0 + slot * TP_STAGE + h * (TP_STAGE / 2), &tm_in,
                          (lc.t.sb + lc.s) * TT_K + 32 * h, lc.t.tile * TT_M, rfull(slot));
        cur_next(lc);
      }
      if (!ok) *fail = 1;
      for (int i = 0; i < R; ++i) {  // the last issue of each slot has landed (bounded)
        const int nis = issued_r > i ? (issued_r - 1 - i) / R + 1 : 0;
        if (nis > 0) tc::mbar_wait(rfull(i), (nis - 1) & 1);
      }
    }
  } else {
    const int qq = warp & 3, hh = warp >> 2, row = qq * 32 + lane;
    float tot[NH];
#pragma unroll
    for (int c = 0; c < NH; ++c) tot[c] = 0.f;
    // thread: trace row `row` of the tile, samples 32 hh .. 32 hh + 31 of each stage (box hh)
    auto convert = [&](int g) -> bool {
      const int slot = g % R;
      if (!tc::mbar_wait_or(rfull(slot), (g / R) & 1, fail)) return false;
      const unsigned rs = ring0 + slot * TP_STAGE + hh * (TP_STAGE / 2) + row * 128;
      float4 v[8];
#pragma unroll
      for (int c = 0; c < 8; ++c)  // 16-byte chunk c of the row sits at c ^ (row % 8)
        asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];"
                     : "=f"(v[c].x), "=f"(v[c].y), "=f"(v[c].z), "=f"(v[c].w)
                     : "r"(rs + (unsigned)((c ^ (row & 7)) << 4)));
      tc::mbar_arrive(rempty(slot));
      // split into bf16 hi / lo while the MMAs of stage g - NA may still read the A tile
      unsigned hi[16], lo[16];
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const __nv_bfloat162 h01 = __floats2bfloat162_rn(v[c].x, v[c].y);
        const __nv_bfloat162 h23 = __floats2bfloat162_rn(v[c].z, v[c].w);
        const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[c].x - f01.x, v[c].y - f01.y);
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[c].z - f23.x, v[c].w - f23.y);
        hi[2 * c] = *reinterpret_cast<const unsigned*>(&h01);
        hi[2 * c + 1] = *reinterpret_cast<const unsigned*>(&h23);
        lo[2 * c] = *reinterpret_cast<const unsigned*>(&l01);
        lo[2 * c + 1] = *reinterpret_cast<const unsigned*>(&l23);
      }
      const bool freed = g < NA || tc::mbar_wait_or(mdone(g), (g / NA - 1) & 1, fail);
      if (!__all_sync(0xffffffffu, freed)) return false;  // the TMEM stores are warp-wide
      tc::tc_fence_after();
      const unsigned at = tmem + ((unsigned)(qq * 32) << 16) + ACOL + (unsigned)((g % NA) * 64 + 16 * hh);
      tc::tmem_st16(at, hi);
      tc::tmem_st16(at + 32, lo);
      tc::tmem_st_wait();
      tc::tc_fence_before();
      tc::mbar_arrive(afull(g));
      return true;
    };
    auto drain = [&](int b) -> bool {  // TMEM block b into the totals
      const bool got = tc::mbar_wait_or(blkd(b & 1), (b >> 1) & 1, fail);
      if (!__all_sync(0xffffffffu, got)) return false;
      tc::tc_fence_after();
      const unsigned base =
          tmem + ((unsigned)(qq * 32) << 16) + (unsigned)((b & 1) * 2 * N + hh * NH);
#pragma unroll
      for (int c0 = 0; c0 < NH; c0 += 16) {
        float x[16], y[16];
        tc::tmem_ld16(base + (unsigned)c0, x);          // hi.hi + lo.hi
        tc::tmem_ld16(base + (unsigned)(N + c0), y);    // hi.lo
#pragma unroll
        for (int i = 0; i < 16; ++i) tot[c0 + i] += x[i] + y[i];
      }
      tc::tc_fence_before();
      tc::mbar_arrive(tempty(b & 1));
      return true;
    };
    auto emit = [&](int tile) {  // a unit's totals into the spectra: components 2 kk, 2 kk + 1
      const int q = tile * TT_M + row;
      if (q < ntr) {
        const int sidx = q / nrec, r = q % nrec;
#pragma unroll
        for (int p = 0; p < NH / 2; ++p) {
          const int kk = hh * (NH / 2) + p;
          if (kk < nf) {
            float2* d = Dh + ((long long)kk * nrec + r) * ld + s0 + sidx;
            const float2 x = make_float2(tot[2 * p], tot[2 * p + 1]);
            if (H == 1)
              *d = x;
            else
              atomicAdd(d, x);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < NH; ++c) tot[c] = 0.f;
    };
    int g = 0, blk = 0, pend = -1, pend_tile = -1;
    for (int i = 0; i < n && ok; ++i) {
      const TpUnit t = tp_unit(u0 + i, H, nst);
      for (int s = 0; s < t.nr; ++s) {
        if (!convert(g)) {
          ok = false;
          break;
        }
        ++g;
        // the block that ended one stage ago; after a unit's last block, its totals go out
        if (pend >= 0) {
          if (!drain(pend)) {
            ok = false;
            break;
          }
          if (pend_tile >= 0) emit(pend_tile);
          pend = -1;
        }
        if ((s + 1) % TT_J == 0 || s == t.nr - 1) {
          pend = blk++;
          pend_tile = s == t.nr - 1 ? t.tile : -1;
        }
      }
    }
    if (ok && pend >= 0) {
      ok = drain(pend);
      if (ok && pend_tile >= 0) emit(pend_tile);
    }
    if (!ok) *fail = 1;
  }
  const bool okall = __syncthreads_and(ok) && !*fail;
  if (!okall && tid == 0) atomicExch(err, 1);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, TCOLS);
}

cudaError_t launch_trace_dft_tc(const float* resid, int ntr, int nt_d, const unsigned char* twt,
                                int nf, int nrec, int ld, int s0, float2* Dh, int* err,
                                int expire, cudaStream_t st) {
  const int N = tt_ncomp(nf);
  const size_t smem = trace_dft_tc_smem(nf);
  const bool vec = (nt_d & 3) == 0 && (reinterpret_cast<uintptr_t>(resid) & 15) == 0;
  const long long tiles = (ntr + TT_M - 1) / TT_M;
  const dim3 grid((unsigned)(tiles * TD_S));
  cudaError_t e = cudaSuccess;
#define EGH_TT_CASE(NN)                                                                        \
  if (N == NN) {                                                                               \
    auto kern = vec ? k_trace_dft_tc<NN, true> : k_trace_dft_tc<NN, false>;                    \
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem))) \
      return e;                                                                                \
    count_launches(1);                                                                         \
    kern<<<grid, 256, smem, st>>>(resid, ntr, nt_d, twt, nf, nrec, ld, s0, Dh, err, expire);   \
    return cudaGetLastError();                                                                 \
  }
  EGH_TT_CASE(32)
  EGH_TT_CASE(64)
  EGH_TT_CASE(96)
  EGH_TT_CASE(128)
#undef EGH_TT_CASE
  return cudaErrorInvalidValue;
}

// Persistent transform: one CTA per SM, at most one per unit.  With two parts per tile the
// spectra of the call's columns are zeroed first (the parts add into them).
cudaError_t launch_trace_tma(const float* resid, int ntr, int nt_d, const unsigned char* twt,
                             int nf, int nrec, int ld, int s0, float2* Dh, int* err, int expire,
                             cudaStream_t st) {
  const int N = tt_ncomp(nf);
  const size_t smem = trace_tma_smem(N);
  auto kern = N == 32 ? k_trace_tma<32> : k_trace_tma<64>;
  cudaError_t e;
  int dev = 0, sms = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return e;
  if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
    return e;
  const int ntile = (ntr + TT_M - 1) / TT_M, nst = (nt_d + TT_K - 1) / TT_K;
  const int H = nst >= 2 ? 2 : 1;
  if (H == 2 &&
      (e = cudaMemset2DAsync(Dh + s0, (size_t)ld * sizeof(float2), 0,
                             (size_t)(ntr / nrec) * sizeof(float2), (size_t)nf * nrec, st)))
    return e;
  CUtensorMap tm;
  if ((e = make_f32_tmap(&tm, resid, ntr, nt_d, 32, TT_M, true))) return e;
  const int grid = (int)std::min<long long>((long long)ntile * H, sms);
  count_launches(1);
  kern<<<grid, TP_EPI + 64, smem, st>>>(tm, ntr, nt_d, twt, nf, nrec, ld, s0, H, Dh, err, expire);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Triangular solves L y = d, L^H x = y for 32 right-hand sides (sources) per block, one block per
// (frequency, column group).  The RHS block lives in shared memory; for each row the dot product
// over earlier rows is split across the eight warps and reduced through shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int TS_W = 8;

__device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(32 * TS_W)
    k_trsm(const float2* __restrict__ Lh, int n, float2* __restrict__ Dh, int ns) {
  extern __shared__ float2 Y[];  // [n][32]
  __shared__ float2 red[TS_W][32];
  const int k = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool valid = col < ns;
  const float2* L = Lh + (long long)k * n * n;
  float2* B = Dh + (long long)k * n * ns;
  for (int i = warp; i < n; i += TS_W)
    Y[i * 32 + lane] = valid ? B[(long long)i * ns + col] : make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    float2 s = make_float2(0.f, 0.f);
    for (int j = warp; j < i; j += TS_W) {
      const float2 p = cmul(L[(long long)i * n + j], Y[j * 32 + lane]);
      s.x += p.x;
      s.y += p.y;
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      float2 t = Y[i * 32 + lane];
#pragma unroll
      for (int w = 0; w < TS_W; ++w) {
        t.x -= red[w][lane].x;
        t.y -= red[w][lane].y;
      }
      const float d = 1.f / L[(long long)i * n + i].x;
      Y[i * 32 + lane] = make_float2(t.x * d, t.y * d);
    }
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {
    float2 s = make_float2(0.f, 0.f);
    for (int j = i + 1 + warp; j < n; j += TS_W) {
      const float2 p = cmulc(L[(long long)j * n + i], Y[j * 32 + lane]);
      s.x += p.x;
      s.y += p.y;
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      float2 t = Y[i * 32 + lane];
#pragma unroll
      for (int w = 0; w < TS_W; ++w) {
        t.x -= red[w][lane].x;
        t.y -= red[w][lane].y;
      }
      const float d = 1.f / L[(long long)i * n + i].x;
      Y[i * 32 + lane] = make_float2(t.x * d, t.y * d);
    }
    __syncthreads();
  }
  if (valid)
    for (int i = warp; i < n; i += TS_W) B[(long long)i * ns + col] = Y[i * 32 + lane];
}

cudaError_t launch_trsm(const float2* Lh, int n, int nf, float2* Dh, int ns, cudaStream_t st) {
  const size_t smem = sizeof(float2) * 32 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((ns + 31) / 32, nf);
  count_launches(1);
  k_trsm<<<grid, 32 * TS_W, smem, st>>>(Lh, n, Dh, ns);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Synthesis: 64 traces x 128 samples per block.  The weighted solutions of the block's traces
// (X[k][trace]) and the twiddles of its time range (T[k][sample]) sit in shared memory; thread
// (g, p) produces samples 4p .. 4p + 3 of traces 8g .. 8g + 7 (per frequency: two 16-byte
// twiddle reads, four broadcast solution reads, 32 packed FP32x2 FMAs).
// Re(X e^{+i theta}) = Re X cos(theta) + Im X (-sin(theta)) with tw = e^{-i theta}.
// ---------------------------------------------------------------------------------------------
constexpr int SY_TR = 64, SY_T = 128, SY_TP = SY_T + 4;

__global__ void __launch_bounds__(256)
    k_synth(const float2* __restrict__ Dh, int nrec, int ld, int s0, int nf,
            const float* __restrict__ w, const float2* __restrict__ tw, int nt_d,
            float* __restrict__ mult, int ntr) {
  extern __shared__ float4 sm4[];
  float2* X = reinterpret_cast<float2*>(sm4);            // [nf][SY_TR]
  float* Tc = reinterpret_cast<float*>(X + SY_TR * nf);  // [nf][SY_TP] cos(theta)
  float* Ts = Tc + nf * SY_TP;                           // [nf][SY_TP] -sin(theta)
  const int tid = threadIdx.x;
  const int q0 = blockIdx.y * SY_TR, t0 = blockIdx.x * SY_T;
  // all gathers in flight at once (cp.async, zero-filled outside), then the weights applied
  for (int e = tid; e < SY_TR * nf; e += 256) {
    const int k = e / SY_TR, rr = e % SY_TR, q = q0 + rr;
    const bool ok = q < ntr;
    cp_async8(X + e, ok ? Dh + ((long long)k * nrec + q % nrec) * ld + s0 + q / nrec : Dh, ok);
  }
  // the block's twiddle rows are one contiguous run of the table: read it in order, transpose
  // on the way into shared memory as separate cos and -sin planes (row length SY_TP keeps the
  // writes at few-way conflicts)
  for (int e = tid; e < nf * SY_T; e += 256) {
    const int tt = e / nf, k = e % nf, t = t0 + tt;
    const bool ok = t < nt_d;
    const float* src = reinterpret_cast<const float*>(ok ? tw + (long long)t0 * nf + e : tw);
    cp_async4(Tc + k * SY_TP + tt, src, ok);
    cp_async4(Ts + k * SY_TP + tt, src + 1, ok);
  }
  cp_async_commit();
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
  for (int e = tid; e < SY_TR * nf; e += 256) {  // the elements this thread copied itself
    const float wk = w[e / SY_TR];
    X[e].x *= wk;
    X[e].y *= wk;
  }
  __syncthreads();
  const int p = tid & 31, g = tid >> 5;
  // acc[m][h] = samples 4p + 2h, 4p + 2h + 1 of trace 8g + m (packed FP32x2, same roundings as
  // the scalar sum Re X cos + Im X (-sin), the sine term first)
  float2 acc[8][2];
#pragma unroll
  for (int m = 0; m < 8; ++m) acc[m][0] = acc[m][1] = make_float2(0.f, 0.f);
  for (int k = 0; k < nf; ++k) {
    const float4 cc = *reinterpret_cast<const float4*>(Tc + k * SY_TP + 4 * p);
    const float4 ss = *reinterpret_cast<const float4*>(Ts + k * SY_TP + 4 * p);
    const float2 c2[2] = {make_float2(cc.x, cc.y), make_float2(cc.z, cc.w)};
    const float2 s2[2] = {make_float2(ss.x, ss.y), make_float2(ss.z, ss.w)};
    const float4* xp = reinterpret_cast<const float4*>(X + k * SY_TR + 8 * g);
#pragma unroll
    for (int h = 0; h < 4; ++h) {
      const float4 xv = xp[h];
      const float2 x[2] = {make_float2(xv.x, xv.y), make_float2(xv.z, xv.w)};
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float2 re = make_float2(x[u].x, x[u].x), im = make_float2(x[u].y, x[u].y);
#pragma unroll
        for (int hh = 0; hh < 2; ++hh)
          acc[2 * h + u][hh] = __ffma2_rn(re, c2[hh], __ffma2_rn(im, s2[hh], acc[2 * h + u][hh]));
      }
    }
  }
  const int tb = t0 + 4 * p;
  const bool vec =
      (nt_d & 3) == 0 && tb + 3 < nt_d && (reinterpret_cast<uintptr_t>(mult) & 15) == 0;
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int q = q0 + 8 * g + m;
    if (q >= ntr) break;
    float* out = mult + (long long)q * nt_d + tb;
    if (vec) {
      *reinterpret_cast<float4*>(out) = make_float4(acc[m][0].x, acc[m][0].y, acc[m][1].x, acc[m][1].y);
    } else {
      const float v[4] = {acc[m][0].x, acc[m][0].y, acc[m][1].x, acc[m][1].y};
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (tb + i < nt_d) out[i] = v[i];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Explicit inverse of the Cholesky factor, W_k = L_k^{-1} (lower triangular), for solves as
// matrix products X = W^H (W D).  Column j of W solves L w = e_j by forward substitution,
// w_i = -(sum_{l=j}^{i-1} L_il w_l) / L_ii.  One warp per (frequency, column): the lanes split
// each row's sum (coalesced reads of row i of L) and the column so far sits in shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int TRI_WARPS = 4;

__global__ void __launch_bounds__(32 * TRI_WARPS)
    k_trtri(const float2* __restrict__ Lh, int n, int nf, float2* __restrict__ Wh) {
  extern __shared__ float2 wcol[];  // [TRI_WARPS][n]
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  const long long t = blockIdx.x * (long long)TRI_WARPS + wp;
  if (t >= (long long)n * nf) return;  // warp-uniform
  const int k = (int)(t / n), j = (int)(t % n);
  const float2* L = Lh + (long long)k * n * n;
  float2* W = Wh + (long long)k * n * n;
  float2* w = wcol + (size_t)wp * n;
  for (int i = lane; i < j; i += 32) W[(long long)i * n + j] = make_float2(0.f, 0.f);
  const float wjj = 1.f / L[(long long)j * n + j].x;
  if (lane == 0) {
    w[j] = make_float2(wjj, 0.f);
    W[(long long)j * n + j] = w[j];
  }
  __syncwarp();
  for (int i = j + 1; i < n; ++i) {
    const float2* Li = L + (long long)i * n;
    float2 acc = make_float2(0.f, 0.f);
    for (int l = j + lane; l < i; l += 32) {
      const float2 a = Li[l], v = w[l];
      acc.x = fmaf(a.x, v.x, fmaf(-a.y, v.y, acc.x));
      acc.y = fmaf(a.x, v.y, fmaf(a.y, v.x, acc.y));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    const float d = -1.f / Li[i].x;
    if (lane == 0) {
      w[i] = make_float2(acc.x * d, acc.y * d);
      W[(long long)i * n + j] = w[i];
    }
    __syncwarp();
  }
}

cudaError_t launch_trtri(const float2* Lh, int n, int nf, float2* Wh, cudaStream_t st) {
  const long long m = (long long)n * nf;
  const size_t smem = (size_t)TRI_WARPS * n * sizeof(float2);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_trtri, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_trtri<<<(unsigned)((m + TRI_WARPS - 1) / TRI_WARPS), 32 * TRI_WARPS, smem, st>>>(Lh, n, nf, Wh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Batched complex products C_k = op(W_k) B_k, op = identity or conjugate transpose, W_k n x n,
// B_k and C_k n x ld (all frequencies in one launch).  32 x 32 output tiles, 32-deep K steps
// staged in shared memory over the triangle's nonzero range; each of the 256 threads computes a
// 2 x 2 block.
// ---------------------------------------------------------------------------------------------
constexpr int CG_T = 32;

template <bool CONJT>
__global__ void __launch_bounds__(256)
    k_cgemm(const float2* __restrict__ Wh, int n, const float2* __restrict__ Bh, int ld,
            float2* __restrict__ Ch, const int* __restrict__ kl) {
  __shared__ float2 As[CG_T][CG_T + 1];  // As[r][kk] = op(W)[row0 + r][k0 + kk]
  __shared__ float2 Bs[CG_T][CG_T + 1];  // Bs[kk][c] = B[k0 + kk][col0 + c]
  const int k = kl ? kl[blockIdx.z] : blockIdx.z;
  const float2* W = Wh + (long long)k * n * n;
  const float2* B = Bh + (long long)k * n * ld;
  float2* C = Ch + (long long)k * n * ld;
  const int row0 = blockIdx.y * CG_T, col0 = blockIdx.x * CG_T;
  const int tid = threadIdx.x, tr = (tid >> 4) * 2, tc = (tid & 15) * 2;
  float2 acc[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) acc[a][b] = make_float2(0.f, 0.f);
  // W is lower triangular (its upper part stored as zeros): rows row0.. of W need k < row0 + 32,
  // rows of W^H need k >= row0
  const int kbeg = CONJT ? row0 : 0, kend = CONJT ? n : min(n, row0 + CG_T);
  for (int k0 = kbeg; k0 < kend; k0 += CG_T) {
    for (int e = tid; e < CG_T * CG_T; e += 256) {
      const int r = e / CG_T, c = e % CG_T;
      float2 a = make_float2(0.f, 0.f);
      if (CONJT) {
        // op(W)[i][kk] = conj(W[kk][i]): read rows of W, coalesced along i
        const int kk = k0 + r, i = row0 + c;
        if (kk < n && i < n) a = W[(long long)kk * n + i];
        As[c][r] = make_float2(a.x, -a.y);
      } else {
        const int i = row0 + r, kk = k0 + c;
        if (i < n && kk < n) a = W[(long long)i * n + kk];
        As[r][c] = a;
      }
      const int kk = k0 + r, cc = col0 + c;
      Bs[r][c] = (kk < n && cc < ld) ? B[(long long)kk * ld + cc] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < CG_T; ++kk) {
      const float2 a0 = As[tr][kk], a1 = As[tr + 1][kk];
      const float2 b0 = Bs[kk][tc], b1 = Bs[kk][tc + 1];
      const float2 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          acc[a][b].x = fmaf(av[a].x, bv[b].x, fmaf(-av[a].y, bv[b].y, acc[a][b].x));
          acc[a][b].y = fmaf(av[a].x, bv[b].y, fmaf(av[a].y, bv[b].x, acc[a][b].y));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = row0 + tr + a, c = col0 + tc + b;
      if (i < n && c < ld) C[(long long)i * ld + c] = acc[a][b];
    }
}

// Q^{-1} = W^H W per frequency (dense Hermitian n x n), the operator of the tensor-core solve.
cudaError_t launch_gram_inverse(const float2* Wh, int n, int nf, float2* Ph, cudaStream_t st) {
  const dim3 grid((n + CG_T - 1) / CG_T, (n + CG_T - 1) / CG_T, nf);
  count_launches(1);
  k_cgemm<true><<<grid, 256, 0, st>>>(Wh, n, Wh, n, Ph, nullptr);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Refinement residual in FP64: R_k = D_k - Q_k X_k, products of the FP32 operands (exact in FP64)
// accumulated in double and rounded once (mixed-precision iterative refinement of the solves).
// One block per (frequency, 32 sources, group of rows); X_k's columns sit in shared memory;
// warp w takes rows w, w + 8, ... of its group; lane = source.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * TS_W)
    k_resid64(const float2* __restrict__ Qh, int n, const float2* __restrict__ Xh,
              const float2* __restrict__ Dh, int ns, float2* __restrict__ Rh,
                 const int* __restrict__ kl) {
  extern __shared__ float2 Xs[];  // [n][32]
  const int k = kl ? kl[blockIdx.y] : blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool valid = col < ns;
  const float2* Q = Qh + (long long)k * n * n;
  const long long off = (long long)k * n * ns;
  for (int i = warp; i < n; i += TS_W)
    Xs[i * 32 + lane] = valid ? Xh[off + (long long)i * ns + col] : make_float2(0.f, 0.f);
  __syncthreads();
  const int rows = (n + gridDim.z - 1) / gridDim.z;
  const int i0 = blockIdx.z * rows, i1 = min(n, i0 + rows);
  for (int i = i0 + warp; i < i1; i += TS_W) {
    double re = 0.0, im = 0.0;
    const float2* q = Q + (long long)i * n;
    for (int j = 0; j < n; ++j) {
      const float2 a = q[j], x = Xs[j * 32 + lane];
      re = fma((double)a.x, (double)x.x, fma(-(double)a.y, (double)x.y, re));
      im = fma((double)a.x, (double)x.y, fma((double)a.y, (double)x.x, im));
    }
    if (valid) {
      const float2 d = Dh[off + (long long)i * ns + col];
      Rh[off + (long long)i * ns + col] = make_float2((float)((double)d.x - re), (float)((double)d.y - im));
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The same residual with FP64-class accuracy from FP32 arithmetic: the compensated dot product
// Dot2 of Ogita, Rump and Oishi ("Accurate sum and dot product", SIAM J. Sci. Comput. 26, 2005).
// Each product a*b is split exactly into p + e (p = fl(a*b), e = fma(a, b, -p)); the p are summed
// with Knuth's TwoSum, whose rounding errors are gathered with the e in a second FP32 word, so
// the result is as accurate as if summed in twice the working precision (about 2^-48 relative to
// sum |q x|) and then rounded.  The GB300 issues FP64 at a small fraction of the FP32 rate, so this
// is the fast route to a residual whose FP32 rounding matches the FP64 one.  Every step uses the
// _rn intrinsics so that no product is contracted into an FMA.  Layout as k_resid64; each warp
// takes two rows per pass so that each solution read serves both.
// ---------------------------------------------------------------------------------------------
__device__ __forceinline__ void dot2_add(float& s, float& c, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = __fmaf_rn(a, b, -p);
  const float t = __fadd_rn(s, p);
  const float bp = __fsub_rn(t, s);
  const float q = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bp)), __fsub_rn(p, bp));
  s = t;
  c = __fadd_rn(c, __fadd_rn(q, e));
}

// The same for a pair of sums at once (real and imaginary parts) in packed FP32x2 instructions:
// element by element the operations and their roundings are those of dot2_add.
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ void dot2_add2(float2& s, float2& c, float2 a, float2 b) {
  const float2 p = __fmul2_rn(a, b);
  const float2 e = __ffma2_rn(a, b, neg2(p));
  const float2 t = __fadd2_rn(s, p);
  const float2 bp = __fadd2_rn(t, neg2(s));
  const float2 q = __fadd2_rn(__fadd2_rn(s, neg2(__fadd2_rn(t, neg2(bp)))), __fadd2_rn(p, neg2(bp)));
  s = t;
  c = __fadd2_rn(c, __fadd2_rn(q, e));
}

__global__ void __launch_bounds__(32 * TS_W)
    k_resid_dot2(const float2* __restrict__ Qh, int n, const float2* __restrict__ Xh,
                 const float2* __restrict__ Dh, int ns, float2* __restrict__ Rh,
                 const int* __restrict__ kl) {
  extern __shared__ float2 Xs[];  // [n][32]
  const int k = kl ? kl[blockIdx.y] : blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool valid = col < ns;
  const float2* Q = Qh + (long long)k * n * n;
  const long long off = (long long)k * n * ns;
  for (int i = warp; i < n; i += TS_W)
    Xs[i * 32 + lane] = valid ? Xh[off + (long long)i * ns + col] : make_float2(0.f, 0.f);
  __syncthreads();
  const int rows = (n + gridDim.z - 1) / gridDim.z;
  const int i0 = blockIdx.z * rows, i1 = min(n, i0 + rows);
  for (int i = i0 + 2 * warp; i < i1; i += 2 * TS_W) {
    const bool two = i + 1 < i1;
    const float2* qa = Q + (long long)i * n;
    const float2* qb = Q + (long long)(two ? i + 1 : i) * n;
    float2 da = make_float2(0.f, 0.f), db = make_float2(0.f, 0.f);
    if (valid) {
      da = Dh[off + (long long)i * ns + col];
      if (two) db = Dh[off + (long long)(i + 1) * ns + col];
    }
    // R = D - Q X: the real part adds (-q.x) x.x then q.y x.y, the imaginary part (-q.x) x.y then
    // (-q.y) x.x; (real, imaginary) sums and their compensations run as packed pairs
    float2 sa = da, ca = make_float2(0.f, 0.f), sb = db, cb = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int j = 0; j < n; ++j) {
      const float2 x = Xs[j * 32 + lane], xs = make_float2(x.y, x.x);
      const float2 a = __ldg(qa + j), b = __ldg(qb + j);
      dot2_add2(sa, ca, make_float2(-a.x, -a.x), x);
      dot2_add2(sa, ca, make_float2(a.y, -a.y), xs);
      dot2_add2(sb, cb, make_float2(-b.x, -b.x), x);
      dot2_add2(sb, cb, make_float2(b.y, -b.y), xs);
    }
    if (valid) {
      Rh[off + (long long)i * ns + col] = __fadd2_rn(sa, ca);
      if (two) Rh[off + (long long)(i + 1) * ns + col] = __fadd2_rn(sb, cb);
    }
  }
}

cudaError_t launch_resid(const float2* Qh, int n, int nf, const float2* Xh, const float2* Dh,
                         int ns, float2* Rh, bool fp64, cudaStream_t st, const int* kl) {
  if (nf < 1) return cudaSuccess;
  const size_t smem = sizeof(float2) * 32 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e = fp64 ? cudaFuncSetAttribute(k_resid64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)
                         : cudaFuncSetAttribute(k_resid_dot2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  // enough blocks for every SM: split the rows of each (frequency, source group)
  const int blocks = ((ns + 31) / 32) * nf;
  const int groups = std::max(1, std::min((n + TS_W - 1) / TS_W, (4 * 152 + blocks - 1) / blocks));
  const dim3 grid((ns + 31) / 32, nf, groups);
  if (fp64)
    k_resid64<<<grid, 32 * TS_W, smem, st>>>(Qh, n, Xh, Dh, ns, Rh, kl);
  else
    k_resid_dot2<<<grid, 32 * TS_W, smem, st>>>(Qh, n, Xh, Dh, ns, Rh, kl);
  return cudaGetLastError();
}

// Diagonal-Hessian baseline: X_k[r][s] = D_k[r][s] / Q_k[r][r] (Q's diagonal is real, >= mu)
__global__ void k_diag_solve(const float2* __restrict__ Qh, int n, float2* __restrict__ Dh, int ns,
                             long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const long long kr = i / ns;  // k * n + r
    const long long k = kr / n, r = kr % n;
    const float q = Qh[(k * n + r) * n + r].x;
    float2 d = Dh[i];
    d.x /= q;
    d.y /= q;
    Dh[i] = d;
  }
}

cudaError_t launch_diag_solve(const float2* Qh, int n, int nf, float2* Dh, int ns, cudaStream_t st) {
  const long long m = (long long)nf * n * ns;
  const int blocks = (int)std::min<long long>((m + 255) / 256, 4 * 152);
  count_launches(1);
  k_diag_solve<<<blocks, 256, 0, st>>>(Qh, n, Dh, ns, m);
  return cudaGetLastError();
}

// X += R (complex, all frequencies and sources)
// X_k += R_k for the frequencies of the list (m = elements per frequency), all when kl is null.
__global__ void k_add_correction(float2* __restrict__ X, const float2* __restrict__ R, long long m,
                                 const int* __restrict__ kl) {
  const long long off = (long long)(kl ? kl[blockIdx.y] : blockIdx.y) * m;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 r = R[off + i];
    float2 x = X[off + i];
    x.x += r.x;
    x.y += r.y;
    X[off + i] = x;
  }
}

cudaError_t launch_add_correction(float2* X, const float2* R, long long m, int nk, cudaStream_t st,
                                  const int* kl) {
  if (nk < 1) return cudaSuccess;
  long long blocks = (m + 255) / 256;
  if (blocks > 512) blocks = 512;
  count_launches(1);
  k_add_correction<<<dim3((unsigned)blocks, (unsigned)nk), 256, 0, st>>>(X, R, m, kl);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Synthesis on the tensor cores: mult[q][t] = sum_c A[q][c] B[t][c] with A[q][2k] = w_k Re X_k,
// A[q][2k+1] = w_k Im X_k (the weighted solutions of trace q) and B[t][2k] = cos(theta),
// B[t][2k+1] = -sin(theta) (host tiles, bf16 hi/lo, K-major 128-byte swizzle).  The components
// come in KC chunks of 64: KC = 1 for 2 nf <= 64 (tiles of 256 samples, two B buffers), KC = 2
// for 2 nf <= 128 (tiles of 128 samples, one B buffer refilled as soon as a tile's MMAs are done,
// while the previous tile drains).  128 traces x 1024 samples per CTA: the threads gather, weight
// and split their solutions into the A tile once, then every sample tile is one bf16x3
// M128 x N(256 or 128) x K(64 KC) product into one of two TMEM buffers, drained by eight warps
// (lane quarter w % 4, column half w / 4) straight to global memory while the next tile's MMAs
// run.  Every wait is bounded.
// ---------------------------------------------------------------------------------------------
constexpr int SC_M = 128;
constexpr int SC_STG = 36;  // row length (floats) of the per-warp 32 x 32 staging tiles
constexpr unsigned SC_CH = SC_M * 128;  // one 64-component chunk of an A plane (hi or lo)
constexpr unsigned SC_B = 65536u;       // one B tile (hi + lo): 2 planes x KC x (256 / KC) x 128 B

__host__ __device__ constexpr int sc_kc(int nf) { return 2 * nf <= 64 ? 1 : 2; }
__host__ __device__ constexpr int sc_n(int kc) { return kc == 1 ? 256 : 128; }  // samples per tile

size_t synth_tc_smem(int kc) {
  // A (2 planes x kc chunks), B buffers (2 for kc = 1, 1 for kc = 2), staging, alignment slack
  return 1024 + 2 * (size_t)kc * SC_CH + (kc == 1 ? 2 : 1) * (size_t)SC_B +
         8 * 32 * SC_STG * sizeof(float);
}

template <bool VEC, int KC>
__global__ void __launch_bounds__(256)
    k_synth_tc(const float2* __restrict__ Dh, int nrec, int ld, int s0, int nf,
               const float* __restrict__ w, const unsigned char* __restrict__ tws, int nt_d,
               float* __restrict__ mult, int ntr, int* __restrict__ err) {
  constexpr int SN = sc_n(KC);          // samples per tile (MMA N)
  constexpr int NB = KC == 1 ? 2 : 1;   // B buffers
  constexpr int SEG = 1024 / SN;        // tiles per CTA
  constexpr unsigned SA = KC * SC_CH;   // one A plane
  extern __shared__ __align__(1024) unsigned char sc_dsm[];
  unsigned char* sm = sc_dsm + ((1024 - (tc::smem_u32(sc_dsm) & 1023)) & 1023);
  __shared__ __align__(8) unsigned long long bars[4];  // bfull[2], mdone[2]
  __shared__ unsigned tslot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int q0 = blockIdx.x * SC_M;
  const int j0 = blockIdx.y * SEG;  // first sample tile of this CTA
  const int ntile = min(SEG, (nt_d + SN - 1) / SN - j0);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto bfull = [&](int i) { return bar0 + 8u * i; };
  auto mdone = [&](int i) { return bar0 + 8u * (2 + i); };
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * SN);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    fail = 0;
    tc::mbar_init_fence();
  }
  const unsigned ah = tc::smem_u32(sm), al = ah + SA;
  auto b_hi = [&](int b) { return tc::smem_u32(sm + 2 * SA + (size_t)b * SC_B); };
  float* stage_all = reinterpret_cast<float*>(sm + 2 * SA + NB * SC_B);  // [8 warps][32][SC_STG]
  // A tile: row m = trace q0 + m, components c = 2k (re), 2k + 1 (im), zero past 2 nf and ntr;
  // the threads of half h take frequencies 16 KC h .. 16 KC h + 16 KC - 1
  {
    const int m = tid & (SC_M - 1), q = q0 + m;
    const int sidx = q / nrec, r = q % nrec;
#pragma unroll 4
    for (int k = (tid >> 7) * 16 * KC; k < (tid >> 7) * 16 * KC + 16 * KC; ++k) {
      float2 x = make_float2(0.f, 0.f);
      if (q < ntr && k < nf) {
        x = Dh[((long long)k * nrec + r) * ld + s0 + sidx];
        const float wk = w[k];
        x.x *= wk;
        x.y *= wk;
      }
      const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
      // chunk k / 32; bytes 4 (k % 32) .. + 3 of row m: 16-byte chunk (k % 32) / 4, offset 4 (k % 4)
      const int kl = k & 31;
      const unsigned off = (unsigned)((k >> 5) * SC_CH + (m >> 3) * 1024 + (m & 7) * 128 +
                                      ((((kl >> 2) ^ (m & 7))) << 4) + ((kl & 3) << 2));
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(ah + off), "r"(*reinterpret_cast<const unsigned*>(&h))
                   : "memory");
      asm volatile("st.shared.u32 [%0], %1;" ::"r"(al + off), "r"(*reinterpret_cast<const unsigned*>(&l))
                   : "memory");
    }
  }
  tc::fence_proxy_async();
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  auto issue_b = [&](int j) {
    tc::mbar_expect_tx(bfull(j % NB), SC_B);
    tc::bulk_g2s(b_hi(j % NB), tws + (size_t)(j0 + j) * SC_B, SC_B, bfull(j % NB));
  };
  if (tid == 0 && ntile > 0) issue_b(0);
  const unsigned idesc = tc::idesc_bf16(SC_M, SN, 0, 0);
  const bool vec = VEC;
  int issued = ntile > 0 ? 1 : 0, waited = 0;
  bool ok = true;
  auto epilogue = [&](int j) {  // TMEM buffer j % 2 -> mult[q][SN (j0 + j) ..]
    const bool got = tc::mbar_wait(mdone(j & 1), (j >> 1) & 1);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      return;
    }
    tc::tc_fence_after();
    const int qq = warp & 3, hh = warp >> 2, lane = tid & 31;
    const unsigned base =
        tmem + ((unsigned)(qq * 32) << 16) + (unsigned)((j & 1) * SN + hh * (SN / 2));
    // each 32 x 32 block goes through this warp's staging tile so that a store instruction
    // writes four full 128-byte rows: lanes 8i .. 8i + 7 cover row 4p + i of pass p
    float* stg = stage_all + warp * (32 * SC_STG);
#pragma unroll 1
    for (int c0 = hh * (SN / 2); c0 < (hh + 1) * (SN / 2); c0 += 32) {
      float v[32];
      tc::tmem_ld32(base + (unsigned)(c0 - hh * (SN / 2)), v);
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(stg + lane * SC_STG + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
      __syncwarp();
      const int t = (j0 + j) * SN + c0 + 4 * (lane & 7);
#pragma unroll
      for (int pp = 0; pp < 8; ++pp) {
        const int rl = 4 * pp + (lane >> 3);
        const int q = q0 + qq * 32 + rl;
        const float4 x = *reinterpret_cast<const float4*>(stg + rl * SC_STG + 4 * (lane & 7));
        if (q < ntr) {
          float* out = mult + (long long)q * nt_d + t;
          if (vec && t + 3 < nt_d) {
            __stcs(reinterpret_cast<float4*>(out), x);
          } else {
            const float xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int i = 0; i < 4; ++i)
              if (t + i < nt_d) out[i] = xv[i];
          }
        }
      }
      __syncwarp();
    }
    tc::tc_fence_before();
  };
  for (int j = 0; j < ntile; ++j) {
    if (tid == 0) {
      // TMEM buffer j % 2 was drained by the epilogue of tile j - 2 (before the last barrier)
      if (!tc::mbar_wait(bfull(j % NB), (j / NB) & 1)) {
        fail = 1;
      } else {
        waited = j + 1;
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)((j & 1) * SN);
        const unsigned bh = b_hi(j % NB), bl = bh + KC * SN * 128;
#pragma unroll
        for (int kc = 0; kc < KC; ++kc)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const unsigned oa = kc * SC_CH + 32u * ks, ob = kc * SN * 128 + 32u * ks;
            const uint64_t dah = tc::sdesc_sw128(ah + oa), dal = tc::sdesc_sw128(al + oa);
            const uint64_t dbh = tc::sdesc_sw128(bh + ob), dbl = tc::sdesc_sw128(bl + ob);
            tc::mma_bf16(dt, dah, dbh, idesc, kc > 0 || ks > 0);
            tc::mma_bf16(dt, dah, dbl, idesc, true);
            tc::mma_bf16(dt, dal, dbh, idesc, true);
          }
        tc::mma_commit(mdone(j & 1));
        // one B buffer: the next tile's twiddles load once this tile's MMAs are done, while
        // the previous tile drains
        if (NB == 1 && j + 1 < ntile) {
          if (!tc::mbar_wait(mdone(j & 1), (j >> 1) & 1)) {
            fail = 1;
          } else {
            issue_b(j + 1);
            issued = j + 2;
          }
        }
      }
    }
    __syncthreads();
    if (fail) {
      ok = false;
      break;
    }
    if (j >= 1) {
      epilogue(j - 1);  // also proves the MMAs of tile j - 1 done: its B buffer is free
      if (!__syncthreads_and(ok)) {
        ok = false;
        break;
      }
    }
    if (NB == 2 && tid == 0 && j + 1 < ntile) {
      if (j == 0 || ok) {
        issue_b(j + 1);
        issued = j + 2;
      }
    }
    __syncthreads();
  }
  if (ok && ntile > 0) epilogue(ntile - 1);
  if (tid == 0) {  // no copy or MMA left in flight (bounded)
    for (int j = waited; j < issued; ++j) tc::mbar_wait(bfull(j % NB), (j / NB) & 1);
    if (waited > 0) tc::mbar_wait(mdone((waited - 1) & 1), ((waited - 1) >> 1) & 1);
  }
  const bool okall = __syncthreads_and(ok) && !fail;
  if (!okall && tid == 0) atomicExch(err, 1);
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * SN);
}

// ---------------------------------------------------------------------------------------------
// Synthesis operands: the A tiles of k_synth_tma as they sit in shared memory, built once per
// call in global memory.  Tile qt holds traces qt * 128 + m; its image is a hi plane and a lo
// plane of KC 64-component chunks each (bf16, K-major, 128-byte swizzle), component 2k =
// Re(w_k D[k][r][s]), 2k + 1 = Im, zero past 2 nf.  One block per (receiver r, 32 sources):
// the spectra are read along the sources (contiguous) and each trace's row is written as
// 16-byte chunks.
// ---------------------------------------------------------------------------------------------
constexpr int SP_SB = 32;  // sources per block of the operand transpose

template <int KC>
__global__ void __launch_bounds__(256)
    k_synth_operands(const float2* __restrict__ Dh, int nrec, int ns, int ld, int s0, int nf,
                     const float* __restrict__ w, unsigned char* __restrict__ img) {
  constexpr int NK = 32 * KC;           // frequencies of the A tile
  constexpr unsigned SA = KC * SC_CH;   // one plane of a tile image
  __shared__ float2 T[NK][SP_SB + 1];
  const int r = blockIdx.x, sb = blockIdx.y * SP_SB, tid = threadIdx.x;
  for (int e = tid; e < NK * SP_SB; e += 256) {
    const int k = e / SP_SB, sl = e % SP_SB, sidx = sb + sl;
    float2 x = make_float2(0.f, 0.f);
    if (k < nf && sidx < ns) {
      const float2 d = Dh[((long long)k * nrec + r) * ld + s0 + sidx];
      const float wk = w[k];
      x = make_float2(d.x * wk, d.y * wk);
    }
    T[k][sl] = x;
  }
  __syncthreads();
  // 16-byte chunk ch of a plane row covers frequencies 4 ch .. 4 ch + 3
  for (int e = tid; e < SP_SB * (NK / 4); e += 256) {
    const int sl = e / (NK / 4), ch = e % (NK / 4), sidx = sb + sl;
    if (sidx >= ns) continue;
    const long long q = (long long)sidx * nrec + r;
    const int m = (int)(q % SC_M);
    unsigned hi[4], lo[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float2 x = T[4 * ch + i][sl];
      const __nv_bfloat162 h = __floats2bfloat162_rn(x.x, x.y);
      const float2 hf = __bfloat1622float2(h);
      const __nv_bfloat162 l = __floats2bfloat162_rn(x.x - hf.x, x.y - hf.y);
      hi[i] = *reinterpret_cast<const unsigned*>(&h);
      lo[i] = *reinterpret_cast<const unsigned*>(&l);
    }
    const int cc = ch & 7;  // chunk within the 64-component block ch / 8
    const size_t off = (size_t)(q / SC_M) * 2 * SA + (size_t)(ch >> 3) * SC_CH + (m >> 3) * 1024 +
                       (m & 7) * 128 + ((cc ^ (m & 7)) << 4);
    *reinterpret_cast<uint4*>(img + off) = make_uint4(hi[0], hi[1], hi[2], hi[3]);
    *reinterpret_cast<uint4*>(img + off + SA) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
  }
}

size_t synth_operands_bytes(int nf, long long ntr) {
  return (size_t)((ntr + SC_M - 1) / SC_M) * 2 * sc_kc(nf) * SC_CH;
}

// ---------------------------------------------------------------------------------------------
// Persistent synthesis into device memory: the same products as k_synth_tc, one CTA per SM over
// an even share of the (trace tile, sample tile) units, roles split by warp.  Warp 8 (one
// thread) loads the twiddle tiles (two buffers) and issues each unit's bf16x3 MMAs into one of
// two TMEM buffers; warps 0-7 fill the A tile of a new trace tile (once the last MMAs that read
// the old one are done), then drain each finished TMEM buffer: a 32 x 32 block per step goes
// through a 128-byte-swizzled staging tile and out with one TMA store (rows past ntr and
// samples past nt_d are clipped by the copy).  mbarriers carry every hand-off; every wait is
// bounded and gives up early once another role has failed.
// ---------------------------------------------------------------------------------------------
constexpr int SP_EPI = 256;  // epilogue threads (warps 0-7); warp 8 issues copies and MMAs

__host__ __device__ constexpr int sp_nstg(int kc) { return kc == 1 ? 2 : 1; }  // staging tiles per warp

size_t synth_tma_smem(int kc) {
  // A (2 planes x kc chunks), 2 B buffers, staging tiles of 4 KB, alignment slack
  return 1024 + 2 * (size_t)kc * SC_CH + 2 * (size_t)SC_B + 8 * (size_t)sp_nstg(kc) * 4096;
}

template <int KC>
__global__ void __launch_bounds__(SP_EPI + 32, 1)
    k_synth_tma(const __grid_constant__ CUtensorMap tm_out, const float2* __restrict__ Dh, int nrec,
                int ld, int s0, int nf, const float* __restrict__ w,
                const unsigned char* __restrict__ tws, int nt_d, int ntr,
                const unsigned char* __restrict__ aimg, int* __restrict__ err) {
  constexpr int SN = sc_n(KC);         // samples per unit (MMA N)
  constexpr unsigned SA = KC * SC_CH;  // one A plane
  constexpr int NSTG = sp_nstg(KC);
  extern __shared__ __align__(1024) unsigned char sp_dsm[];
  unsigned char* sm = sp_dsm + ((1024 - (tc::smem_u32(sp_dsm) & 1023)) & 1023);
  // bfull[2], mdone[2], tempty[2], afull (A filled by warps 0-7), aload (A copied from aimg)
  __shared__ __align__(8) unsigned long long bars[8];
  __shared__ unsigned tslot;
  __shared__ int fail_s;
  volatile int* fail = &fail_s;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nj = (nt_d + SN - 1) / SN;  // sample tiles per trace tile
  const long long U = (long long)((ntr + SC_M - 1) / SC_M) * nj;
  const long long u0 = U * blockIdx.x / gridDim.x;
  const int n = (int)(U * (blockIdx.x + 1) / gridDim.x - u0);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto bfull = [&](int i) { return bar0 + 8u * i; };
  auto mdone = [&](int i) { return bar0 + 8u * (2 + i); };
  auto tempty = [&](int i) { return bar0 + 8u * (4 + i); };
  const unsigned afull = bar0 + 48u, aload = bar0 + 56u;
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * SN);
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    tc::mbar_init(tempty(0), SP_EPI);
    tc::mbar_init(tempty(1), SP_EPI);
    tc::mbar_init(afull, SP_EPI);
    tc::mbar_init(aload, 1);
    fail_s = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  const unsigned ah = tc::smem_u32(sm), al = ah + SA;
  auto b_hi = [&](int b) { return tc::smem_u32(sm + 2 * SA + (size_t)b * SC_B); };
  const unsigned stg0 = tc::smem_u32(sm + 2 * SA + 2 * SC_B);
  bool ok = true;
  if (warp == 8) {
    if (lane == 0 && n > 0) {
      auto issue_b = [&](int i) {
        const int j = (int)((u0 + i) % nj);
        tc::mbar_expect_tx(bfull(i & 1), SC_B);
        tc::bulk_g2s(b_hi(i & 1), tws + (size_t)j * SC_B, SC_B, bfull(i & 1));
      };
      const unsigned idesc = tc::idesc_bf16(SC_M, SN, 0, 0);
      int issued_b = 0, waited_b = 0, issued_m = 0, tiles = 0;
      long long qt_prev = -1;
      issue_b(0);
      issued_b = 1;
      if (n > 1) {
        issue_b(1);
        issued_b = 2;
      }
      for (int i = 0; i < n; ++i) {
        const long long qt = (u0 + i) / nj;
        if (qt != qt_prev) {  // the A tile of this trace tile
          if (aimg) {
            // copied from its image once the previous tile's last MMAs are done
            if (i >= 1 && !tc::mbar_wait_or(mdone((i - 1) & 1), ((i - 1) >> 1) & 1, fail)) {
              ok = false;
              break;
            }
            tc::mbar_expect_tx(aload, 2 * SA);
            tc::bulk_g2s(ah, aimg + (size_t)qt * 2 * SA, 2 * SA, aload);
            if (!tc::mbar_wait_or(aload, tiles & 1, fail)) {
              ok = false;
              break;
            }
          } else if (!tc::mbar_wait_or(afull, tiles & 1, fail)) {  // filled by warps 0-7
            ok = false;
            break;
          }
          ++tiles;
          qt_prev = qt;
        }
        if (!tc::mbar_wait_or(bfull(i & 1), (i >> 1) & 1, fail)) {
          ok = false;
          break;
        }
        waited_b = i + 1;
        // TMEM buffer i % 2 was drained by the epilogue of unit i - 2
        if (i >= 2 && !tc::mbar_wait_or(tempty(i & 1), ((i - 2) >> 1) & 1, fail)) {
          ok = false;
          break;
        }
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)((i & 1) * SN);
        const unsigned bh = b_hi(i & 1), bl = bh + KC * SN * 128;
#pragma unroll
        for (int kc = 0; kc < KC; ++kc)
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const unsigned oa = kc * SC_CH + 32u * ks, ob = kc * SN * 128 + 32u * ks;
            const uint64_t dah = tc::sdesc_sw128(ah + oa), dal = tc::sdesc_sw128(al + oa);
            const uint64_t dbh = tc::sdesc_sw128(bh + ob), dbl = tc::sdesc_sw128(bl + ob);
            tc::mma_bf16(dt, dah, dbh, idesc, kc > 0 || ks > 0);
            tc::mma_bf16(dt, dah, dbl, idesc, true);
            tc::mma_bf16(dt, dal, dbh, idesc, true);
          }
        tc::mma_commit(mdone(i & 1));
        issued_m = i + 1;
        // B buffer i % 2 takes unit i + 2's twiddles once this unit's MMAs are done
        if (i + 2 < n) {
          if (!tc::mbar_wait_or(mdone(i & 1), (i >> 1) & 1, fail)) {
            ok = false;
            break;
          }
          issue_b(i + 2);
          issued_b = i + 3;
        }
      }
      if (!ok) *fail = 1;
      // leave no copy or MMA in flight (bounded)
      for (int i = waited_b; i < issued_b; ++i) tc::mbar_wait(bfull(i & 1), (i >> 1) & 1);
      if (issued_m > 0) tc::mbar_wait(mdone((issued_m - 1) & 1), ((issued_m - 1) >> 1) & 1);
    }
  } else {
    // A tile of trace tile qt: row m = trace qt * 128 + m, components c = 2k (re), 2k + 1 (im),
    // zero past 2 nf and ntr; the threads of half h take frequencies 16 KC h .. 16 KC h + 16 KC - 1
    auto fill_a = [&](long long qt) {
      const int m = tid & (SC_M - 1);
      const long long q = qt * SC_M + m;
      const int sidx = (int)(q / nrec), r = (int)(q % nrec);
      const int kb = (tid >> 7) * 16 * KC;
      float2 x[16 * KC];
#pragma unroll
      for (int i = 0; i < 16 * KC; ++i) {
        const int k = kb + i;
        x[i] = make_float2(0.f, 0.f);
        if (q < ntr && k < nf) {
          const float2 d = Dh[((long long)k * nrec + r) * ld + s0 + sidx];
          const float wk = w[k];
          x[i] = make_float2(d.x * wk, d.y * wk);
        }
      }
#pragma unroll
      for (int i = 0; i < 16 * KC; ++i) {
        const int k = kb + i;
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[i].x, x[i].y);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(x[i].x - hf.x, x[i].y - hf.y);
        const int kl = k & 31;
        const unsigned off = (unsigned)((k >> 5) * SC_CH + (m >> 3) * 1024 + (m & 7) * 128 +
                                        ((((kl >> 2) ^ (m & 7))) << 4) + ((kl & 3) << 2));
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(ah + off), "r"(*reinterpret_cast<const unsigned*>(&h))
                     : "memory");
        asm volatile("st.shared.u32 [%0], %1;" ::"r"(al + off), "r"(*reinterpret_cast<const unsigned*>(&l))
                     : "memory");
      }
      tc::fence_proxy_async();
      tc::mbar_arrive(afull);
    };
    if (n > 0 && !aimg) fill_a(u0 / nj);
    const int qq = warp & 3, hh = warp >> 2;
    int cnt = 0;  // staging tiles used by this warp
    for (int i = 0; i < n; ++i) {
      const long long u = u0 + i, qt = u / nj;
      const int j = (int)(u % nj);
      if (!tc::mbar_wait_or(mdone(i & 1), (i >> 1) & 1, fail)) {
        ok = false;
        break;
      }
      tc::tc_fence_after();
      // the next unit starts a new trace tile: refill A now that its last MMAs are done
      if (!aimg && i + 1 < n && (u + 1) / nj != qt) fill_a(qt + 1);
      const unsigned base =
          tmem + ((unsigned)(qq * 32) << 16) + (unsigned)((i & 1) * SN + hh * (SN / 2));
#pragma unroll 1
      for (int c0 = 0; c0 < SN / 2; c0 += 32) {
        float v[32];
        tc::tmem_ld32(base + (unsigned)c0, v);
        if (cnt >= NSTG) {  // the staging tile's previous store has read it
          if (lane == 0) tc::bulk_wait_read<NSTG - 1>();
          __syncwarp();
        }
        const unsigned sb = stg0 + (unsigned)((warp * NSTG + cnt % NSTG) * 4096);
#pragma unroll
        for (int k = 0; k < 8; ++k)
          asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(
                           sb + lane * 128 + ((k ^ (lane & 7)) << 4)),
                       "f"(v[4 * k]), "f"(v[4 * k + 1]), "f"(v[4 * k + 2]), "f"(v[4 * k + 3])
                       : "memory");
        tc::fence_proxy_async();
        __syncwarp();
        if (lane == 0) {
          // a box that starts past the last sample or trace writes nothing: not issued (the
          // group is still committed, so that the staging tiles' group count stays in step)
          const int t = j * SN + hh * (SN / 2) + c0, q = (int)(qt * SC_M) + qq * 32;
          if (t < nt_d && q < ntr) tc::tma_store_2d(&tm_out, sb, t, q);
          tc::bulk_commit();
        }
        ++cnt;
      }
      tc::tc_fence_before();
      tc::mbar_arrive(tempty(i & 1));
    }
    if (!ok) *fail = 1;
    if (lane == 0) tc::bulk_wait_all();
  }
  const bool okall = __syncthreads_and(ok) && !*fail;
  if (!okall && tid == 0) atomicExch(err, 1);
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * SN);
}

// Synthesis twiddle tiles: for every sample tile (256 samples for 2 nf <= 64, else 128), a hi and
// a lo plane, each [KC chunks of 64 components][tile samples][64 components] bf16 in the K-major
// 128-byte swizzle (row t, component c of chunk kc at byte kc * rows * 128 + (t/8)*1024 +
// (t%8)*128 + (((2c/16) ^ (t%8)) * 16) + 2c%16); component 2k = cos(2 pi f_k t dt), 2k + 1 =
// -sin(2 pi f_k t dt) with the phase reduced as 2 pi frac(f_k t dt) in double precision; hi =
// bf16(w), lo = bf16(w - hi); components >= 2 nf and samples >= nt are zero.
std::vector<unsigned char> synth_twiddle_tiles(const std::vector<double>& f, double dt, int nt) {
  const int nf = (int)f.size();
  const int kc_n = sc_kc(nf), sn = sc_n(kc_n);
  const int ntile = (nt + sn - 1) / sn;
  std::vector<unsigned char> out((size_t)ntile * SC_B, 0);
  for (int t = 0; t < nt; ++t) {
    unsigned char* hi = out.data() + (size_t)(t / sn) * SC_B;
    unsigned char* lo = hi + (size_t)kc_n * sn * 128;
    const int r = t % sn;
    for (int k = 0; k < nf && 2 * k + 1 < 64 * kc_n; ++k) {
      double ph = f[k] * (double)t * dt;
      ph -= std::floor(ph);
      const double a = 2.0 * M_PI * ph;
      const double v[2] = {std::cos(a), -std::sin(a)};
      for (int qq = 0; qq < 2; ++qq) {
        const int c = 2 * k + qq, kc = c / 64, cl = c % 64;
        const size_t off = (size_t)kc * sn * 128 + (size_t)(r >> 3) * 1024 + (r & 7) * 128 +
                           ((((2 * cl) >> 4) ^ (r & 7)) << 4) + ((2 * cl) & 15);
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v[qq]);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)(v[qq] - (double)__bfloat162float(h)));
        std::memcpy(hi + off, &h, 2);
        std::memcpy(lo + off, &l, 2);
      }
    }
  }
  return out;
}

// Tensor map of a [rows][cols] fp32 array (row pitch cols) for box_cols x box_rows boxes, with
// or without the 128-byte swizzle.
cudaError_t make_f32_tmap(CUtensorMap* tm, const void* base, long long rows, long long cols,
                          int box_cols, int box_rows, bool swizzle) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    cudaError_t e =
        cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q);
    if (e != cudaSuccess) return e;
    if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
    enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  const cuuint64_t str[1] = {(cuuint64_t)cols * 4};
  const cuuint32_t box[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(base), dims, str,
                         box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         swizzle ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_NONE,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t launch_synth_tc(const float2* Dh, int nrec, int ns, int ld, int s0, int nf,
                            const float* w, const unsigned char* tws, int nt_d, float* mult,
                            int* err, cudaStream_t st, bool dev_out, unsigned char* scratch,
                            size_t scratch_bytes) {
  const int ntr = nrec * ns;
  const int kc = sc_kc(nf), sn = sc_n(kc);
  const bool vec = (nt_d & 3) == 0 && (reinterpret_cast<uintptr_t>(mult) & 15) == 0;
  cudaError_t e;
  if (vec && dev_out && ntr > 0) {
    // device memory: the persistent kernel with TMA stores, one CTA per SM; its A tiles come
    // from operand images built first when a scratch buffer of their size is given
    CUtensorMap tm;
    if ((e = make_f32_tmap(&tm, mult, ntr, nt_d, 32, 32, true))) return e;
    unsigned char* aimg = nullptr;
    if (scratch && scratch_bytes >= synth_operands_bytes(nf, ntr) &&
        (reinterpret_cast<uintptr_t>(scratch) & 15) == 0) {
      aimg = scratch;
      const dim3 pg((unsigned)nrec, (unsigned)((ns + SP_SB - 1) / SP_SB));
      count_launches(1);
      if (kc == 1)
        k_synth_operands<1><<<pg, 256, 0, st>>>(Dh, nrec, ns, ld, s0, nf, w, aimg);
      else
        k_synth_operands<2><<<pg, 256, 0, st>>>(Dh, nrec, ns, ld, s0, nf, w, aimg);
      if ((e = cudaGetLastError())) return e;
    }
    const size_t smem = synth_tma_smem(kc);
    auto kern = kc == 1 ? k_synth_tma<1> : k_synth_tma<2>;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
      return e;
    int dev = 0, sms = 0;
    if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
      return e;
    const long long units = (long long)((ntr + SC_M - 1) / SC_M) * ((nt_d + sn - 1) / sn);
    const int grid = (int)std::min<long long>(units, sms);
    count_launches(1);
    kern<<<grid, SP_EPI + 32, smem, st>>>(tm, Dh, nrec, ld, s0, nf, w, tws, nt_d, ntr, aimg, err);
    return cudaGetLastError();
  }
  const size_t smem = synth_tc_smem(kc);
  auto kern = kc == 1 ? (vec ? k_synth_tc<true, 1> : k_synth_tc<false, 1>)
                      : (vec ? k_synth_tc<true, 2> : k_synth_tc<false, 2>);
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  const int ntile = (nt_d + sn - 1) / sn, seg = 1024 / sn;
  const dim3 grid((ntr + SC_M - 1) / SC_M, (ntile + seg - 1) / seg);
  kern<<<grid, 256, smem, st>>>(Dh, nrec, ld, s0, nf, w, tws, nt_d, mult, ntr, err);
  return cudaGetLastError();
}

cudaError_t launch_synth(const float2* Dh, int nrec, int ns, int ld, int s0, int nf, const float* w,
                         const float2* tw, int nt_d, float* mult, cudaStream_t st,
                         const unsigned char* tws, int* err, bool dev_out, unsigned char* scratch,
                         size_t scratch_bytes) {
  if (nf > NFMAX) return cudaErrorInvalidValue;
  if (tws && err && 2 * nf <= 128)
    return launch_synth_tc(Dh, nrec, ns, ld, s0, nf, w, tws, nt_d, mult, err, st, dev_out, scratch,
                           scratch_bytes);
  const int ntr = nrec * ns;
  const size_t smem = sizeof(float2) * (size_t)nf * SY_TR + 2 * sizeof(float) * (size_t)nf * SY_TP;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((nt_d + SY_T - 1) / SY_T, (ntr + SY_TR - 1) / SY_TR);
  count_launches(1);
  k_synth<<<grid, 256, smem, st>>>(Dh, nrec, ld, s0, nf, w, tw, nt_d, mult, ntr);
  return cudaGetLastError();
}

}  // namespace egh
