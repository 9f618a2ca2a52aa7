// Per-frequency Hessians on the tensor cores (eq. Qmatrix with S S^T replaced by its
// frequency-domain blocks; Section "Direct Hessian-inverse computation", Algorithm 2):
//   H_k[i][j] = sum_x ghat_i(w_k, x) conj(ghat_j(w_k, x)).
// With M_k = [Re ghat_0; Im ghat_0; Re ghat_1; ...] (2 nrec rows, G columns) and the real symmetric
// C = M_k M_k^T:
//   Re H[i][j] = C[2i][2j] + C[2i+1][2j+1],   Im H[i][j] = C[2i+1][2j] - C[2i][2j+1].
//
// C is formed in 128 x 256 blocks (64 x 128 receivers x re/im; 128 x 128 at the last panel)
// covering exactly the panel pairs on and above the diagonal, by tcgen05 `kind::f16` MMAs in
// bf16x3: each entry of M_k is stored by the transform's
// last chunk as hi = bf16(g), lo = bf16(g - hi), and C = Hi Hi^T + Hi Lo^T + Lo Hi^T accumulates in
// FP32 in TMEM (the dropped Lo Lo^T and the split are ~2^-17 relative).  Operands arrive by 5-D TMA
// boxes of 32 points x 64 receivers x re/im that land as 128 rows of 64 bytes in the K-major
// 64-byte-swizzled layout the MMA reads, so the kernel does no conversion.  The grid
// sum is split into `splits` ranges; each CTA writes its FP32 tile to a workspace and a second
// kernel adds the splits (in double) and forms Q_k.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "egh_internal.cuh"
#include "tc.cuh"

namespace egh {

constexpr int GC_M = 128;            // block rows of C (64 receivers x re/im)
constexpr int GC_N = 256;            // block columns of C (128 receivers x re/im)
constexpr int GC_P = 64;   // points per operand block of the blocked layout
constexpr int GC_K = 32;   // points per stage: one 64-byte bf16 row (64-byte swizzle)
constexpr int GC_ST = 4;   // stages in flight (4 x 48 KB: the copies run three stages ahead)
constexpr unsigned GC_BOX = 128u * GC_K * 2;  // one operand box: 64 receivers x re/im = 128 rows
constexpr unsigned GC_STAGE = 6 * GC_BOX;  // A hi, A lo (1 box each), B hi, B lo (2 boxes each)

// Blocks (ta, j) of C: rows of 64-receiver panel ta (128 rows), columns of panels ta + 2j and
// ta + 2j + 1 (256 columns; a "half" block when the second panel is past the last), j = 0, 1, ...
// -- exactly the panel pairs on and above the diagonal.  Block (ta, 0) is "inner": its A panel is
// the first half of its B panels.
__host__ __device__ inline int gram_tc_panels64(int nrec) { return (nrec + 63) / 64; }
__host__ __device__ inline int gram_tc_blocks_before(int ta, int n64) {
  int s = 0;
  for (int t = 0; t < ta; ++t) s += (n64 - t + 1) / 2;
  return s;
}
__host__ __device__ int gram_tc_blocks(int nrec) {
  const int n64 = gram_tc_panels64(nrec);
  return gram_tc_blocks_before(n64, n64);
}

size_t gram_tc_workspace_floats(int nrec, int nf, int splits) {
  return (size_t)splits * nf * gram_tc_blocks(nrec) * GC_M * GC_N;
}

size_t gram_tc_smem() { return 1024 + (size_t)GC_ST * GC_STAGE; }

// Tensor map of the bf16 transforms, blocked by 64 points as
// ghb[nf][G/64][hi/lo][nrec x re/im][64], for boxes {32 points, 128 rows (64 receivers x re/im),
// 1 plane, 1 block, 1 frequency} with the 64-byte swizzle: every box is 128 runs of 64 bytes
// 128 bytes apart (one half of a contiguous 16 KB block).
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
  const cuuint64_t rows = 2ull * nrec;
  const cuuint64_t dims[5] = {(cuuint64_t)GC_P, rows, 2, (cuuint64_t)(G / GC_P), (cuuint64_t)nf};
  const cuuint64_t str[4] = {GC_P * 2, rows * GC_P * 2, 2 * rows * GC_P * 2,
                             (cuuint64_t)(G / GC_P) * 2 * rows * GC_P * 2};
  const cuuint32_t box[5] = {GC_K, 128, 1, 1, 1};
  const cuuint32_t es[5] = {1, 1, 1, 1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, str, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// The Gram's bf16 operands from FP32 transforms gh[nrec][nf][re/im][G]: hi = bf16(g),
// lo = bf16(g - hi), blocked by 64 points as ghb[nf][G/64][hi/lo][nrec x re/im][64] (the layout the
// transform's last chunk writes, from the same values).
__global__ void k_gh_to_ghb(const float* __restrict__ gh, int nrec, int nf, long long G,
                            __nv_bfloat16* __restrict__ ghb) {
  const long long total = (long long)nrec * nf * 2 * G;
  const long long rows = 2LL * nrec;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < total;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t % G, c2 = (t / G) % (2LL * nf), r = t / (2LL * nf * G);
    const float v = gh[t];
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const __nv_bfloat16 l = __float2bfloat16_rn(v - __bfloat162float(h));
    __nv_bfloat16* q = ghb + (((c2 >> 1) * (G >> 6) + (p >> 6)) * 2 * rows + 2 * r + (c2 & 1)) * 64 +
                       (p & 63);
    q[0] = h;
    q[rows * 64] = l;
  }
}

cudaError_t launch_gh_to_ghb(const float* gh, int nrec, int nf, long long G, __nv_bfloat16* ghb,
                             cudaStream_t st) {
  const long long total = (long long)nrec * nf * 2 * G;
  const long long blocks = std::min<long long>((total + 255) / 256, 152LL * 16);
  count_launches(1);
  k_gh_to_ghb<<<(unsigned)blocks, 256, 0, st>>>(gh, nrec, nf, G, ghb);
  return cudaGetLastError();
}

__device__ __forceinline__ void tma_load_5d(unsigned dst, const void* tmap, int c0, int c1, int c2,
                                            int c3, int c4, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.5d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, "
      "%3, %4, %5, %6}], [%7];" ::"r"(dst),
      "l"(tmap), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar)
      : "memory");
}

// One CTA: block (ta, tb) of C at frequency k over points [p0, p1), as M128 x N256 MMAs (each
// A row group read from shared memory serves 256 columns, which halves the operand traffic per
// product against square 128 x 128 tiles).  Warp 8 (one thread) issues the copies and the MMAs
// over a GC_ST-stage ring.  The tensor core's FP32 accumulation of a long sum drifts (its
// rounding is not round-to-nearest: about 2^-24 relative per accumulation, measured 1e-3 over
// 87 000 points), so the MMAs accumulate into one of two 256-column TMEM buffers for blocks of
// GC_J stages only, and warps 0..7 (lane quarter w % 4, column half w / 4) drain each finished
// block into FP32 register totals with round-to-nearest adds while the MMAs fill the other
// buffer.  Stages of 32 points (48 KB) keep four in the ring, the copies three stages ahead of
// the MMAs (measured against two 96 KB stages of 64 points: 9.6 -> 8.1 ms at 231 receivers x
// 26 frequencies).  Every wait is bounded (on expiry: error flag, bounded drain of the copies in
// flight, TMEM freed, CTA leaves).
constexpr int GC_J = 8 * (GC_P / GC_K);  // stages per TMEM accumulation block (96 accumulations)

// K-major shared-memory descriptor of the 64-byte swizzle (8-row groups 512 bytes apart)
__device__ __forceinline__ uint64_t gc_desc(unsigned saddr) { return tc::sdesc_sw64(saddr); }

__global__ void __launch_bounds__(288)
    k_gram_tc(const __grid_constant__ CUtensorMap tmap, int nrec, long long split_len, long long G,
              float* __restrict__ part, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sm = dsm + ((1024 - (tc::smem_u32(dsm) & 1023)) & 1023);
  // full[GC_ST], empty[GC_ST], blockdone[2], drained[2]
  __shared__ __align__(8) unsigned long long bars[2 * GC_ST + 4];
  __shared__ unsigned tslot;
  __shared__ int fail;
  const int blkid = blockIdx.x, k = blockIdx.y, sp = blockIdx.z, nf = gridDim.y;
  const int n64 = gram_tc_panels64(nrec);
  int ta = 0;
  while (ta + 1 < n64 && gram_tc_blocks_before(ta + 1, n64) <= blkid) ++ta;
  const int bp = ta + 2 * (blkid - gram_tc_blocks_before(ta, n64));  // first B panel
  const bool inner = bp == ta;         // the A panel is the first half of the B panels
  const bool half = bp + 1 >= n64;     // one B panel only: N = 128
  const long long p0 = (long long)sp * split_len;
  const long long p1 = min(G, p0 + split_len);
  const int nst = p1 > p0 ? (int)((p1 - p0 + GC_K - 1) / GC_K) : 0;
  const int nblk = (nst + GC_J - 1) / GC_J;
  const int tid = threadIdx.x, warp = tid >> 5;
  if (warp == 0) tc::tmem_alloc(&tslot, 2 * GC_N);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (GC_ST + i); };
  auto blockdone = [&](int i) { return bar0 + 8u * (2 * GC_ST + i); };
  auto drained = [&](int i) { return bar0 + 8u * (2 * GC_ST + 2 + i); };
  if (tid == 0) {
    for (int i = 0; i < 2 * GC_ST + 2; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    tc::mbar_init(drained(0), 256);
    tc::mbar_init(drained(1), 256);
    fail = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  // stage buffer: [A_hi][A_lo][B_hi: 2 boxes][B_lo: 2 boxes]
  auto stage_addr = [&](int b) { return tc::smem_u32(sm + (size_t)b * GC_STAGE); };
  if (warp == 8) {
    if (tid == 256) {
      const unsigned idesc = tc::idesc_bf16(GC_M, half ? GC_N / 2 : GC_N, 0, 0);
      auto issue = [&](int s) {
        const int b = s % GC_ST;
        const int stg = (int)(p0 / GC_P) + s / (GC_P / GC_K);  // 64-point block
        const int xo = GC_K * (s % (GC_P / GC_K));               // its half (64-byte rows)
        const unsigned base = stage_addr(b);
        tc::mbar_expect_tx(full(b), (unsigned)((inner ? 0 : 2) + (half ? 2 : 4)) * GC_BOX);
        for (int hl = 0; hl < 2; ++hl) {
          if (!inner) tma_load_5d(base + hl * GC_BOX, &tmap, xo, 2 * 64 * ta, hl, stg, k, full(b));
          for (int h = 0; h < (half ? 1 : 2); ++h)
            tma_load_5d(base + (2 + 2 * hl + h) * GC_BOX, &tmap, xo, 2 * 64 * (bp + h), hl, stg, k,
                        full(b));
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
        const unsigned dt = tmem + (unsigned)((blk & 1) * GC_N);
        const unsigned bh = stage_addr(b) + 2 * GC_BOX, bl = stage_addr(b) + 4 * GC_BOX;
        // an inner block's A rows are the first 128 B rows
        const unsigned ah = inner ? bh : stage_addr(b);
        const unsigned al = inner ? bl : ah + GC_BOX;
#pragma unroll
        for (int ks = 0; ks < GC_K / 16; ++ks) {
          const unsigned o = 32u * ks;
          const uint64_t dah = gc_desc(ah + o), dal = gc_desc(al + o);
          const uint64_t dbh = gc_desc(bh + o), dbl = gc_desc(bl + o);
          tc::mma_bf16(dt, dah, dbh, idesc, !(first && ks == 0));
          tc::mma_bf16(dt, dah, dbl, idesc, true);
          tc::mma_bf16(dt, dal, dbh, idesc, true);
        }
        tc::mma_commit(empty(b));
        if (s % GC_J == GC_J - 1 || s == nst - 1) tc::mma_commit(blockdone(blk & 1));
        // refill the previous stage's buffer (its MMAs were issued one stage earlier, so the
        // tensor pipe keeps this stage's MMAs queued while the thread waits for them)
        if (s >= 1 && issued < nst) {
          const int pb = (s - 1) % GC_ST;
          if (!tc::mbar_wait(empty(pb), ((s - 1) / GC_ST) & 1)) {
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
    // warps 0..7: TMEM lanes 32 (w % 4) .. = rows of the block, columns 128 (w / 4) ..
    const int q = warp & 3, h = warp >> 2;
    float tot[128];
#pragma unroll
    for (int c = 0; c < 128; ++c) tot[c] = 0.f;
    bool ok = true;
    const bool idle = half && h == 1;  // columns past the last panel: nothing to drain
    for (int blk = 0; blk < nblk; ++blk) {
      const bool got = tc::mbar_wait(blockdone(blk & 1), (blk >> 1) & 1);
      if (!__all_sync(0xffffffffu, got && !fail)) {  // warp-uniform: TMEM loads are collective
        ok = false;
        break;
      }
      tc::tc_fence_after();
      if (!idle) {
        const unsigned base =
            tmem + ((unsigned)(q * 32) << 16) + (unsigned)((blk & 1) * GC_N + h * 128);
#pragma unroll
        for (int c0 = 0; c0 < 128; c0 += 32) {
          float v[32];
          tc::tmem_ld32(base + (unsigned)c0, v);
#pragma unroll
          for (int i = 0; i < 32; ++i) tot[c0 + i] += v[i];
        }
      }
      tc::tc_fence_before();
      tc::mbar_arrive(drained(blk & 1));
    }
    if (ok && !fail && !idle) {
      const int row = q * 32 + (tid & 31);
      float* out = part +
                   (((long long)sp * nf + k) * gram_tc_blocks(nrec) + blkid) * (GC_M * GC_N) +
                   (long long)row * GC_N + h * 128;
#pragma unroll
      for (int i = 0; i < 128; i += 4)
        *reinterpret_cast<float4*>(out + i) = make_float4(tot[i], tot[i + 1], tot[i + 2], tot[i + 3]);
    } else if (!(ok && !fail) && (tid & 31) == 0) {
      atomicExch(err, 1);
    }
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, 2 * GC_N);
}

int gram_tc_splits(int nrec, int nf, long long G) {
  // one CTA per SM (shared memory); about sixteen waves of short point ranges keep the CTAs of
  // one frequency close together in the grid sum, so that their shared panels meet in L2
  // (measured on 231 receivers x 26 frequencies: 6 splits 11.1 ms, 16 splits 10.5 ms)
  const long long blocks = (long long)gram_tc_blocks(nrec) * nf;
  long long s = (16LL * 152 + blocks - 1) / blocks;
  s = std::max(1LL, std::min(s, G / (16LL * GC_P)));
  return (int)s;
}

cudaError_t launch_gram_tc(const CUtensorMap& tmap, int nrec, int nf, long long G, int splits,
                           float* part, int* err, cudaStream_t st) {
  if (G % GC_P != 0 || splits < 1) return cudaErrorInvalidValue;
  long long split_len = (G + splits - 1) / splits;
  split_len = (split_len + GC_P - 1) / GC_P * GC_P;
  const size_t smem = gram_tc_smem();
  cudaError_t e =
      cudaFuncSetAttribute(k_gram_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_gram_tc<<<dim3(gram_tc_blocks(nrec), nf, splits), 288, smem, st>>>(tmap, nrec, split_len, G,
                                                                       part, err);
  return cudaGetLastError();
}

// C[a][b] summed over splits (in double), read from the block that holds (a, b) or, below the
// diagonal blocks, (b, a) (C is symmetric).
__device__ inline double ctc_entry(const float* part, int a, int b, int k, int nf, int n64,
                                   int nblocks, int splits) {
  if (a / GC_M > b / GC_M) {
    const int t = a;
    a = b;
    b = t;
  }
  const int pa = a / GC_M, pb = b / GC_M;
  const int blk = gram_tc_blocks_before(pa, n64) + (pb - pa) / 2;
  const long long off = (long long)(a % GC_M) * GC_N + ((pb - pa) & 1) * GC_M + (b % GC_M);
  double sum = 0.0;
  for (int s = 0; s < splits; ++s)
    sum += part[(((long long)s * nf + k) * nblocks + blk) * (GC_M * GC_N) + off];
  return sum;
}

__global__ void k_gram_tc_finish(const float* __restrict__ part, int nrec, int nf, int splits,
                                 float2* __restrict__ Qh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  const int k = blockIdx.z;
  if (j >= nrec) return;
  const int n64 = gram_tc_panels64(nrec), nblocks = gram_tc_blocks(nrec);
  const int a = min(i, j), b = max(i, j);
  const double rr = ctc_entry(part, 2 * a, 2 * b, k, nf, n64, nblocks, splits);
  const double ii = ctc_entry(part, 2 * a + 1, 2 * b + 1, k, nf, n64, nblocks, splits);
  double im = 0.0;
  if (a != b)
    im = ctc_entry(part, 2 * a + 1, 2 * b, k, nf, n64, nblocks, splits) -
         ctc_entry(part, 2 * a, 2 * b + 1, k, nf, n64, nblocks, splits);
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
