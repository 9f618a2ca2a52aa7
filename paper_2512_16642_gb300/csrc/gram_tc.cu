// Per-frequency Hessians on the tensor cores (eq. Qmatrix with S S^T replaced by its
// frequency-domain blocks; Section "Direct Hessian-inverse computation", Algorithm 2):
//   H_k[i][j] = sum_x ghat_i(w_k, x) conj(ghat_j(w_k, x)).
// With M_k = [Re ghat_0; Im ghat_0; Re ghat_1; ...] (2 nrec rows, G columns) and the real symmetric
// C = M_k M_k^T:
//   Re H[i][j] = C[2i][2j] + C[2i+1][2j+1],   Im H[i][j] = C[2i+1][2j] - C[2i][2j+1].
//
// C is formed in 128 x 128 tiles (64 receivers x re/im per tile edge) on and above the tile
// diagonal by tcgen05 `kind::f16` MMAs in bf16x3: each entry of M_k is stored by the transform's
// last chunk as hi = bf16(g), lo = bf16(g - hi), and C = Hi Hi^T + Hi Lo^T + Lo Hi^T accumulates in
// FP32 in TMEM (the dropped Lo Lo^T and the split are ~2^-17 relative).  Operands arrive by 5-D TMA
// boxes {64 points, hi|lo, re/im, 1 frequency, 64 receivers} that land as 128 rows of 128 bytes in
// the K-major 128-byte-swizzled layout the MMA reads, so the kernel does no conversion.  The grid
// sum is split into `splits` ranges; each CTA writes its FP32 tile to a workspace and a second
// kernel adds the splits (in double) and forms Q_k.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "egh_internal.cuh"
#include "tc.cuh"

namespace egh {

constexpr int GC_T = 128;            // tile edge (rows of M_k)
constexpr int GC_P = 64;             // points per stage (one 128-byte bf16 row)
constexpr int GC_ST = 3;             // stages in flight
constexpr unsigned GC_BOX = 16384;   // one operand box: 128 rows x 128 bytes

__host__ __device__ int gram_tc_tiles(int nrec) { return (2 * nrec + GC_T - 1) / GC_T; }

size_t gram_tc_workspace_floats(int nrec, int nf, int splits) {
  const int nt = gram_tc_tiles(nrec);
  return (size_t)splits * nf * ((size_t)nt * (nt + 1) / 2) * GC_T * GC_T;
}

size_t gram_tc_smem() { return 1024 + (size_t)GC_ST * 4 * GC_BOX; }

// Tensor map of the bf16 transforms ghb[nrec][nf][re/im][hi/lo][G] for boxes
// {64 points, 1 plane, 2 (re/im), 1 frequency, 64 receivers} with the 128-byte swizzle.
cudaError_t make_ghb_tmap(CUtensorMap* tm, void* base, long long G, int nf, int nrec) {
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
  const cuuint64_t dims[5] = {(cuuint64_t)G, 2, 2, (cuuint64_t)nf, (cuuint64_t)nrec};
  const cuuint64_t str[4] = {(cuuint64_t)G * 2, (cuuint64_t)G * 4, (cuuint64_t)G * 8,
                             (cuuint64_t)G * 8 * nf};
  const cuuint32_t box[5] = {GC_P, 1, 2, 1, GC_T / 2};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, str, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

__device__ __forceinline__ void tma_load_5d(unsigned dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, int c4, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// One CTA: tile pair (ta <= tb) of frequency k over points [p0, p1).  Warp 4 (one thread) issues
// the copies and the MMAs over a GC_ST-stage ring.  The tensor core's FP32 accumulation of a long
// sum drifts (its rounding is not round-to-nearest: about 2^-24 relative per accumulation,
// measured 1e-3 over 87 000 points), so the MMAs accumulate into one of two TMEM buffers for
// blocks of GC_J stages only, and warps 0..3 drain each finished block into FP32 register totals
// with round-to-nearest adds while the MMAs fill the other buffer.  Every wait is bounded (on
// expiry: error flag, bounded drain of the copies in flight, TMEM freed, CTA leaves).
constexpr int GC_J = 8;  // stages per TMEM accumulation block (96 accumulations)

__global__ void __launch_bounds__(160)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, int ntile, long long split_len, long long G,
              float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sm = dsm + ((1024 - (tc::smem_u32(dsm) & 1023)) & 1023);
  // full[GC_ST], empty[GC_ST], blockdone[2], drained[2]
  __shared__ __align__(8) unsigned long long bars[2 * GC_ST + 4];
  __shared__ unsigned tslot;
  __shared__ int fail;
  const int pair = blockIdx.x, k = blockIdx.y, sp = blockIdx.z, nf = gridDim.y;
  int ta = 0, rem = pair;
  while (rem >= ntile - ta) {
    rem -= ntile - ta;
    ++ta;
  }
  const int tb = ta + rem;
  const bool diag = ta == tb;
  const long long p0 = (long long)sp * split_len;
  const long long p1 = min(G, p0 + split_len);
  const int nst = p1 > p0 ? (int)((p1 - p0 + GC_P - 1) / GC_P) : 0;
  const int nblk = (nst + GC_J - 1) / GC_J;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 256);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (GC_ST + i); };
  auto blockdone = [&](int i) { return bar0 + 8u * (2 * GC_ST + i); };
  auto drained = [&](int i) { return bar0 + 8u * (2 * GC_ST + 2 + i); };
  if (tid == 0) {
    for (int i = 0; i < 2 * GC_ST + 2; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    tc::mbar_init(drained(0), 128);
    tc::mbar_init(drained(1), 128);
    fail = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  // stage buffer: [A_hi][A_lo][B_hi][B_lo], 16 KB each (B is A on diagonal tiles)
  auto buf_addr = [&](int b, int which) {
    return tc::smem_u32(sm + ((size_t)b * 4 + which) * GC_BOX);
  };
  if (warp == 4) {
    if (tid == 128) {
      const unsigned idesc = tc::idesc_bf16(GC_T, GC_T, 0, 0);
      auto issue = [&](int s) {
        const int b = s % GC_ST;
        const int p = (int)(p0 + (long long)s * GC_P);
        tc::mbar_expect_tx(full(b), (diag ? 2u : 4u) * GC_BOX);
        for (int hl = 0; hl < 2; ++hl) {
          tma_load_5d(buf_addr(b, hl), &tmap, p, hl, 0, k, ta * (GC_T / 2), full(b));
          if (!diag) tma_load_5d(buf_addr(b, 2 + hl), &tmap, p, hl, 0, k, tb * (GC_T / 2), full(b));
        }
      };
      int issued = 0, landed = 0;
      bool ok = true;
      for (; issued < min(nst, GC_ST); ++issued) issue(issued);
      for (int s = 0; s < nst && ok; ++s) {
        const int b = s % GC_ST;
        const int blk = s / GC_J;
        const bool first = s % GC_J == 0;
        // a block reuses the TMEM buffer of block blk - 2 once the drain warps have read it
        if (first && blk >= 2 && !tc::mbar_wait(drained(blk & 1), ((blk >> 1) - 1) & 1)) {
          ok = false;
          break;
        }
        if (!tc::mbar_wait(full(b), (s / GC_ST) & 1)) {
          ok = false;
          break;
        }
        landed = s + 1;
        tc::tc_fence_after();
        const unsigned dt = tmem + (unsigned)((blk & 1) * GC_T);
        const unsigned ah = buf_addr(b, 0), al = buf_addr(b, 1);
        const unsigned bh = diag ? ah : buf_addr(b, 2), bl = diag ? al : buf_addr(b, 3);
#pragma unroll
        for (int ks = 0; ks < GC_P / 16; ++ks) {
          const unsigned o = 32u * ks;
          const uint64_t dah = tc::sdesc_sw128(ah + o), dal = tc::sdesc_sw128(al + o);
          const uint64_t dbh = tc::sdesc_sw128(bh + o), dbl = tc::sdesc_sw128(bl + o);
          tc::mma_bf16(dt, dah, dbh, idesc, !(first && ks == 0));
          tc::mma_bf16(dt, dah, dbl, idesc, true);
          tc::mma_bf16(dt, dal, dbh, idesc, true);
        }
        tc::mma_commit(empty(b));
        if (s % GC_J == GC_J - 1 || s == nst - 1) tc::mma_commit(blockdone(blk & 1));
        if (issued < nst) {  // the next stage to issue reuses this stage's buffer
          if (!tc::mbar_wait(empty(b), (s / GC_ST) & 1)) {
            ok = false;
            break;
          }
          issue(issued);
          ++issued;
        }
      }
      if (!ok) {
        fail = 1;
        atomicExch(err, 1);
        for (int s = landed; s < issued; ++s) tc::mbar_wait(full(s % GC_ST), (s / GC_ST) & 1);
        // wake the drain warps: every MMA issued so far completes before these arrivals
        tc::mma_commit(blockdone(0));
        tc::mma_commit(blockdone(1));
      }
    }
    __syncwarp();
  } else {
    // warps 0..3: TMEM lanes 32 w .. 32 w + 31 = rows of the tile; totals in registers
    float tot[GC_T];
#pragma unroll
    for (int c = 0; c < GC_T; ++c) tot[c] = 0.f;
    bool ok = true;
    for (int blk = 0; blk < nblk; ++blk) {
      const bool got = tc::mbar_wait(blockdone(blk & 1), (blk >> 1) & 1);
      if (!__all_sync(0xffffffffu, got && !fail)) {  // warp-uniform: TMEM loads are collective
        ok = false;
        break;
      }
      tc::tc_fence_after();
      const unsigned base = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)((blk & 1) * GC_T);
#pragma unroll
      for (int c0 = 0; c0 < GC_T; c0 += 32) {
        float v[32];
        tc::tmem_ld32(base + (unsigned)c0, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) tot[c0 + i] += v[i];
      }
      tc::tc_fence_before();
      tc::mbar_arrive(drained(blk & 1));
    }
    if (ok && !fail) {
      const int npairs = ntile * (ntile + 1) / 2;
      float* out = part + (((long long)sp * nf + k) * npairs + pair) * (GC_T * GC_T) +
                   (long long)tid * GC_T;  // row tid of the tile (TMEM lane)
#pragma unroll
      for (int i = 0; i < GC_T; i += 4)
        *reinterpret_cast<float4*>(out + i) = make_float4(tot[i], tot[i + 1], tot[i + 2], tot[i + 3]);
    } else if (tid == 0) {
      atomicExch(err, 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 256);
}

int gram_tc_splits(int nrec, int nf, long long G) {
  const int nt = gram_tc_tiles(nrec);
  const long long tiles = (long long)nt * (nt + 1) / 2 * nf;
  long long s = (3LL * 152 + tiles - 1) / tiles;
  s = std::max(1LL, std::min(s, G / (16LL * GC_P)));
  return (int)s;
}

cudaError_t launch_gram_tc(const CUtensorMap& tmap, int nrec, int nf, long long G, int splits,
                           float* part, int* err, cudaStream_t st) {
  if (G % GC_P != 0 || splits < 1) return cudaErrorInvalidValue;
  const int nt = gram_tc_tiles(nrec);
  const int npairs = nt * (nt + 1) / 2;
  long long split_len = (G + splits - 1) / splits;
  split_len = (split_len + GC_P - 1) / GC_P * GC_P;
  const size_t smem = gram_tc_smem();
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_gram_tc<<<dim3(npairs, nf, splits), 160, smem, st>>>(tmap, nt, split_len, G, part, err);
  return cudaGetLastError();
}

// C[a][b] summed over splits (in double), read from the tile pair with ta <= tb (C is symmetric).
__device__ inline double ctc_entry(const float* part, int a, int b, int k, int nf, int ntile,
                                   int npairs, int splits) {
  if (a / GC_T > b / GC_T) {
    const int t = a;
    a = b;
    b = t;
  }
  const int ta = a / GC_T, tb = b / GC_T;
  const int pair = ta * ntile - ta * (ta - 1) / 2 + (tb - ta);
  const long long off = (long long)(a % GC_T) * GC_T + (b % GC_T);
  double sum = 0.0;
  for (int s = 0; s < splits; ++s)
    sum += part[(((long long)s * nf + k) * npairs + pair) * (GC_T * GC_T) + off];
  return sum;
}

__global__ void k_gram_tc_finish(const float* __restrict__ part, int nrec, int nf, int splits,
                                 float2* __restrict__ Qh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  const int k = blockIdx.z;
  if (j >= nrec) return;
  const int ntile = gram_tc_tiles(nrec);
  const int npairs = ntile * (ntile + 1) / 2;
  const int a = min(i, j), b = max(i, j);
  const double rr = ctc_entry(part, 2 * a, 2 * b, k, nf, ntile, npairs, splits);
  const double ii = ctc_entry(part, 2 * a + 1, 2 * b + 1, k, nf, ntile, npairs, splits);
  double im = 0.0;
  if (a != b)
    im = ctc_entry(part, 2 * a + 1, 2 * b, k, nf, ntile, npairs, splits) -
         ctc_entry(part, 2 * a, 2 * b + 1, k, nf, ntile, npairs, splits);
  // entry (a, b) with a <= b; (b, a) is its conjugate
  Qh[((long long)k * nrec + i) * nrec + j] = make_float2((float)(rr + ii), (float)(i <= j ? im : -im));
}

cudaError_t launch_gram_tc_finish(const float* part, int nrec, int nf, int splits, float2* Qh,
                                  cudaStream_t st) {
  dim3 grid((nrec + 127) / 128, nrec, nf);
  count_launches(1);
  k_gram_tc_finish<<<grid, 128, 0, st>>>(part, nrec, nf, splits, Qh);
  return cudaGetLastError();
}

}  // namespace egh
