// The per-frequency multi-source solve as one dense complex product on the tensor cores
// (eq. Qsystemfreq: X_k = Q_k^{-1} D_k for all sources at once, with Q_k^{-1} = W_k^H W_k formed
// from the inverse Cholesky factor once per factorisation):
//   C_k = A_k B_k,   A_k [n][n], B_k [n][ld], C_k [n][ld] complex64 (row-major).
//
// FP32-class products from bf16 tensor-core MMAs: every entry of A and B is split into three bf16
// terms, x = x0 + x1 + x2 (x0 = bf16(x), x1 = bf16(x - x0), x2 = bf16(x - x0 - x1); 24 bits of
// the significand), and each real product sum_k a b keeps the six term products down to 2^-16
// relative (x2 y0, x1 y1, x0 y2, x1 y0, x0 y1, x0 y0; the dropped ones are 2^-24).  The complex
// product accumulates three real ones, Re A Re B, Re A Im B + Im A Re B and Im A Im B, into three
// adjacent TMEM accumulators: a term's B re and B im planes form one 128-row operand, so Re A x
// [Re B | Im B] and Im A x [Re B | Im B] are two MMAs of width 128, the second offset by one
// accumulator.  The tensor core's FP32 accumulation is not rounded to nearest (the Gram's
// accumulators drifted by about 2^-24 per accumulation), so (1) within a stage the small term
// products are accumulated first and the large x0 y0 ones last, which keeps the drift near one ulp
// of the stage's sum per large accumulation, and (2) each stage's sums leave TMEM for FP32 register
// totals added with round-to-nearest, two accumulator sets alternating so that the MMAs of a stage
// run while the previous stage's sums are read.
//
// One CTA: 128 rows x 64 columns of C of one frequency, K in stages of 32 (K-major operand tiles
// of 64-byte rows in the 64-byte swizzle, as the Gram's), 8 warps.  The threads load the next
// stage into registers while the current one's MMAs run, split it and write the 12 operand planes
// (A and B, re and im, three terms); one thread issues the MMAs.  Every wait is bounded; on expiry
// the CTA records the error flag, lets its MMAs finish and leaves (its output is not written).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>

#include "egh_internal.cuh"
#include "tc.cuh"

namespace egh {

namespace {

constexpr int CM_M = 128, CM_N = 64, CM_K = 32;
constexpr unsigned CM_AP = CM_M * 64;                 // one A plane: 128 rows x 64 bytes
constexpr unsigned CM_BP = CM_N * 64;                 // one B plane: 64 rows x 64 bytes
constexpr unsigned CM_STAGE = 6 * CM_AP + 6 * CM_BP;  // A re/im x 3 terms, B re/im x 3 terms
constexpr int CM_ACC = 3 * CM_N;                      // TMEM columns of one accumulator set

size_t cmm_smem() { return 1024 + 2 * (size_t)CM_STAGE; }

// byte offset of 16-byte chunk ch (0..3) of row r in a K-major tile of 64-byte rows, 64-byte swizzle
__device__ __forceinline__ unsigned sw64_off(int r, int ch) {
  return (unsigned)((r >> 3) * 512 + (r & 7) * 64 + ((ch ^ ((r >> 1) & 3)) << 4));
}

// three-term bf16 split of 8 values into planes t0, t1, t2 (one 16-byte chunk each)
__device__ __forceinline__ void split3(const float (&x)[8], uint4& t0, uint4& t1, uint4& t2) {
  unsigned w0[4], w1[4], w2[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float a = x[2 * i], b = x[2 * i + 1];
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(a, b);
    const float2 f0 = __bfloat1622float2(h0);
    const float ra = a - f0.x, rb = b - f0.y;  // exact (Sterbenz: |r| <= 2^-8 |x|)
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(ra, rb);
    const float2 f1 = __bfloat1622float2(h1);
    const __nv_bfloat162 h2 = __floats2bfloat162_rn(ra - f1.x, rb - f1.y);
    w0[i] = *reinterpret_cast<const unsigned*>(&h0);
    w1[i] = *reinterpret_cast<const unsigned*>(&h1);
    w2[i] = *reinterpret_cast<const unsigned*>(&h2);
  }
  t0 = make_uint4(w0[0], w0[1], w0[2], w0[3]);
  t1 = make_uint4(w1[0], w1[1], w1[2], w1[3]);
  t2 = make_uint4(w2[0], w2[1], w2[2], w2[3]);
}

__device__ __forceinline__ void sts128(unsigned addr, uint4 v) {
  asm volatile("st.shared.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}

__global__ void __launch_bounds__(256, 1)
    k_cmm_tc(const float2* __restrict__ Ah, int n, const float2* __restrict__ Bh, int ld,
             float2* __restrict__ Ch, const int* __restrict__ kl, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char cm_dsm[];
  unsigned char* sm = cm_dsm + ((1024 - (tc::smem_u32(cm_dsm) & 1023)) & 1023);
  __shared__ __align__(8) unsigned long long bars[4];  // mdone[2] (operand buffers), acc[2] (sets)
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int k = kl ? kl[blockIdx.z] : blockIdx.z;
  const int m0 = blockIdx.y * CM_M, c0 = blockIdx.x * CM_N;
  const float2* A = Ah + (long long)k * n * n;
  const float2* B = Bh + (long long)k * n * ld;
  float2* C = Ch + (long long)k * n * ld;
  const int nst = (n + CM_K - 1) / CM_K;
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * CM_ACC <= 256 ? 256 : 512);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto mdone = [&](int i) { return bar0 + 8u * i; };
  auto accd = [&](int i) { return bar0 + 8u * (2 + i); };
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  // stage b: planes [A re 0,1,2][A im 0,1,2][B re 0][B im 0][B re 1][B im 1][B re 2][B im 2]: a
  // term's B re and B im planes are rows 0-63 and 64-127 of one 128-row K-major tile
  auto plane_a = [&](int b, int ri, int t) {
    return tc::smem_u32(sm + (size_t)b * CM_STAGE + (unsigned)(3 * ri + t) * CM_AP);
  };
  auto plane_b = [&](int b, int ri, int t) {
    return tc::smem_u32(sm + (size_t)b * CM_STAGE + 6 * CM_AP + (unsigned)(2 * t + ri) * CM_BP);
  };
  // this thread's pieces of a stage: A rows ra, ra + 64 (chunk ca: 8 consecutive k, 8 float2);
  // B column cb (chunk kb: 8 consecutive k, 8 float2)
  const int ra = tid >> 2, ca = tid & 3;
  const int cb = tid & 63, kb = tid >> 6;
  float2 pa[2][8];
  float2 pb[8];
  auto load = [&](int s) {
    const int k0 = s * CM_K;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = m0 + ra + 64 * h;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int kk = k0 + 8 * ca + j;
        pa[h][j] = (i < n && kk < n) ? A[(long long)i * n + kk] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int kk = k0 + 8 * kb + j;
      const int c = c0 + cb;
      pb[j] = (kk < n && c < ld) ? B[(long long)kk * ld + c] : make_float2(0.f, 0.f);
    }
  };
  auto convert = [&](int b) {
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int r = ra + 64 * h;
      float re[8], im[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        re[j] = pa[h][j].x;
        im[j] = pa[h][j].y;
      }
      const unsigned off = sw64_off(r, ca);
      uint4 t0, t1, t2;
      split3(re, t0, t1, t2);
      sts128(plane_a(b, 0, 0) + off, t0);
      sts128(plane_a(b, 0, 1) + off, t1);
      sts128(plane_a(b, 0, 2) + off, t2);
      split3(im, t0, t1, t2);
      sts128(plane_a(b, 1, 0) + off, t0);
      sts128(plane_a(b, 1, 1) + off, t1);
      sts128(plane_a(b, 1, 2) + off, t2);
    }
    {
      float re[8], im[8];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        re[j] = pb[j].x;
        im[j] = pb[j].y;
      }
      const unsigned off = sw64_off(cb, kb);
      uint4 t0, t1, t2;
      split3(re, t0, t1, t2);
      sts128(plane_b(b, 0, 0) + off, t0);
      sts128(plane_b(b, 0, 1) + off, t1);
      sts128(plane_b(b, 0, 2) + off, t2);
      split3(im, t0, t1, t2);
      sts128(plane_b(b, 1, 0) + off, t0);
      sts128(plane_b(b, 1, 1) + off, t1);
      sts128(plane_b(b, 1, 2) + off, t2);
    }
  };
  // warp w reads TMEM lanes 32 (w % 4) .. (its rows) and columns 32 (w / 4) .. of each accumulator
  const int qq = warp & 3, hh = warp >> 2;
  float trr[32], tii[32], tim[32];
#pragma unroll
  for (int i = 0; i < 32; ++i) trr[i] = tii[i] = tim[i] = 0.f;
  bool ok = true;
  auto drain = [&](int s) {  // add accumulator set s % 2 (stage s) into the totals
    const bool got = tc::mbar_wait(accd(s & 1), (s >> 1) & 1);
    if (!__all_sync(0xffffffffu, got)) {
      ok = false;
      return;
    }
    tc::tc_fence_after();
    // accumulator set: [0, N) Re A Re B, [N, 2N) Re A Im B + Im A Re B, [2N, 3N) Im A Im B
    const unsigned base = tmem + ((unsigned)(qq * 32) << 16) + (unsigned)((s & 1) * CM_ACC + hh * 32);
    float v[32];
    tc::tmem_ld32(base, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) trr[i] += v[i];
    tc::tmem_ld32(base + CM_N, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) tim[i] += v[i];
    tc::tmem_ld32(base + 2 * CM_N, v);
#pragma unroll
    for (int i = 0; i < 32; ++i) tii[i] += v[i];
    tc::tc_fence_before();
  };
  const unsigned idesc = tc::idesc_bf16(CM_M, CM_N, 0, 0), idesc2 = tc::idesc_bf16(CM_M, 2 * CM_N, 0, 0);
  int issued = 0;  // stages whose MMAs were issued (thread 0)
  if (nst > 0) load(0);
  for (int s = 0; s < nst; ++s) {
    const int b = s & 1;
    // operand buffer b was last read by the MMAs of stage s - 2 (block-uniform decision)
    const bool freed = s < 2 || tid != 0 || tc::mbar_wait(mdone(b), ((s - 2) >> 1) & 1);
    if (!__syncthreads_and(freed)) {
      ok = false;
      break;
    }
    convert(b);
    if (s + 1 < nst) load(s + 1);
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::tc_fence_after();
      const unsigned d = tmem + (unsigned)(b * CM_ACC);
      // term products smallest first (i + j = 2, then 1, then 0), both K steps of the stage.
      // Re A x [Re B | Im B] -> columns [0, 2N) (Re Re, then Re Im into the imaginary sums);
      // Im A x [Re B | Im B] -> columns [N, 3N) (Im Re onto the imaginary sums, Im Im).  The
      // very first Im A product writes [2N, 3N) fresh, so it is issued as two N-wide MMAs.
      const int ti[6] = {2, 1, 0, 1, 0, 0}, tj[6] = {0, 1, 2, 0, 1, 0};
#pragma unroll
      for (int p = 0; p < 6; ++p) {
#pragma unroll
        for (int ks = 0; ks < CM_K / 16; ++ks) {
          const unsigned o = 32u * ks;
          const bool first = p == 0 && ks == 0;
          const uint64_t are = tc::sdesc_sw64(plane_a(b, 0, ti[p]) + o);
          const uint64_t aim = tc::sdesc_sw64(plane_a(b, 1, ti[p]) + o);
          const uint64_t bri = tc::sdesc_sw64(plane_b(b, 0, tj[p]) + o);  // [Re B | Im B]
          tc::mma_bf16(d, are, bri, idesc2, !first);
          if (first) {
            const uint64_t bim = tc::sdesc_sw64(plane_b(b, 1, tj[p]) + o);
            tc::mma_bf16(d + CM_N, aim, bri, idesc, true);       // Im A Re B onto Re A Im B
            tc::mma_bf16(d + 2 * CM_N, aim, bim, idesc, false);  // Im A Im B, fresh
          } else {
            tc::mma_bf16(d + CM_N, aim, bri, idesc2, true);
          }
        }
      }
      tc::mma_commit(mdone(b));
      tc::mma_commit(accd(b));
      issued = s + 1;
    }
    // the previous stage's sums leave TMEM while this stage's MMAs run
    if (s >= 1) drain(s - 1);
    if (!__syncthreads_and(ok)) {
      ok = false;
      break;
    }
  }
  if (ok && nst > 0) drain(nst - 1);
  // no MMA in flight when the CTA leaves (bounded): the last commit covers the earlier ones
  if (tid == 0 && issued > 0) tc::mbar_wait(mdone((issued - 1) & 1), ((issued - 1) >> 1) & 1);
  const bool okall = __syncthreads_and(ok);
  if (!okall) {
    if (tid == 0) atomicExch(err, 1);
  } else {
    const int i = m0 + qq * 32 + lane;
    if (i < n) {
      float2* row = C + (long long)i * ld + c0 + hh * 32;
#pragma unroll
      for (int j = 0; j < 32; ++j)
        if (c0 + hh * 32 + j < ld) row[j] = make_float2(trr[j] - tii[j], tim[j]);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * CM_ACC <= 256 ? 256 : 512);
}

}  // namespace

cudaError_t launch_cmm_tc(const float2* A, int n, int nk, const float2* B, int ld, float2* C,
                          const int* kl, int* err, cudaStream_t st) {
  if (nk < 1 || n < 1 || ld < 1) return cudaSuccess;
  if (!err) return cudaErrorInvalidValue;
  const size_t smem = cmm_smem();
  cudaError_t e = cudaFuncSetAttribute(k_cmm_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((ld + CM_N - 1) / CM_N), (unsigned)((n + CM_M - 1) / CM_M), (unsigned)nk);
  count_launches(1);
  k_cmm_tc<<<grid, 256, smem, st>>>(A, n, B, ld, C, kl, err);
  return cudaGetLastError();
}

}  // namespace egh
