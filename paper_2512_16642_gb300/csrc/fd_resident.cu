// Resident finite-difference solver for the Green-function batches (Section "Direct
// Hessian-inverse computation": one wave-equation solve per receiver, eq. wave_eq; the scheme is
// the one of fd.cu, the same operations in the same order, so both give identical levels).
//
// The per-step kernel of fd.cu re-reads two wavefield levels from L2 and writes one back at every
// step.  Here a batch's state stays on the chip for a whole chunk of steps: the padded grid is
// split into one tile per SM (a cooperative launch, so every block is resident), and each block
// keeps both levels of its tile for every receiver pair of the batch in shared memory, with a
// 4-point halo on each side.  After each step a block publishes the 4 boundary rows and columns
// of the new level to a small exchange buffer in global memory (L2) and raises its step counter;
// it then waits for the counters of its (up to four) neighbours and copies their strips into its
// halo.  The eighth-order Laplacian is a cross, so corners are never exchanged.  Only the
// snapshots the transform reads, and the state at the chunk's ends, reach DRAM.
//
// Work inside a block: a unit is (receiver pair, 4 adjacent columns, a segment of SR rows); its
// thread marches down the segment with the z first differences in registers, as fd.cu does, and
// reads the x neighbours from shared memory.  Rows of shared memory are stored as two planes of
// float4 (even and odd float4 slots) so that the threads of one quarter-warp, which take adjacent
// column quads, read adjacent 16-byte words.
//
// Every wait on another block is bounded: on expiry the block records the error flag and an
// abort flag that every other block's wait also watches, so the whole grid returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <climits>

#include "egh_internal.cuh"
#include "tc.cuh"

namespace egh {

namespace {

constexpr int RES_MAXT = 384;  // threads per block at most (a thread takes several units beyond)

__device__ __forceinline__ float2 rsub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}

__device__ __forceinline__ unsigned rbf2(__nv_bfloat162 v) { return *reinterpret_cast<unsigned*>(&v); }

__device__ __forceinline__ void rsplit(float a, float b, unsigned& hi, unsigned& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const float2 r = rsub2(make_float2(a, b), hf);
  hi = rbf2(h);
  lo = rbf2(__floats2bfloat162_rn(r.x, r.y));
}

// the first-difference Laplacian of fd.cu (same operation order)
__device__ __forceinline__ float2 rlap2(const float2 (&dz)[8], const float2* e, const float2 (&cz)[4],
                                        const float2 (&cx)[4]) {
  float2 l = __fmul2_rn(cz[0], rsub2(dz[4], dz[3]));
  l = __ffma2_rn(cz[1], rsub2(dz[5], dz[2]), l);
  l = __ffma2_rn(cz[2], rsub2(dz[6], dz[1]), l);
  l = __ffma2_rn(cz[3], rsub2(dz[7], dz[0]), l);
  l = __ffma2_rn(cx[0], rsub2(e[4], e[3]), l);
  l = __ffma2_rn(cx[1], rsub2(e[5], e[2]), l);
  l = __ffma2_rn(cx[2], rsub2(e[6], e[1]), l);
  l = __ffma2_rn(cx[3], rsub2(e[7], e[0]), l);
  return l;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct ResArgs {
  float2* lev;        // [3][pslot][F] state slots (level t in slot t mod 3)
  long long F;        // float2 per level per pair
  int pslot;          // pairs per state slot
  long long org;      // padded point (0, 0) inside a level
  int NZ, NX, PX;
  const float2* coef; // (c1, c3) per padded point, pitched like a level
  int np;             // pairs of this batch (<= geometry P)
  int ta, nsteps;     // levels ta .. ta + nsteps - 1 are computed
  int t0, decim, sbase;  // snapshot of level t: ring slot sbase + (t - t0) / decim if t % decim == 0
  __nv_bfloat16* snap;   // ring base (hi plane of slot 0), or null for no snapshots
  long long sslot, splane, srec;  // elements per ring slot, hi -> lo plane, per receiver
  float4* xbuf;       // [2][tiles][P][SB] exchange strips
  int* flags;         // [tiles] steps completed in this launch (zeroed before the launch)
  int* abort_flag;    // set by a block whose wait ran out (zeroed before the launch)
  int* err;           // the context's error flag
  int expire;         // test hook: block 0's first wait runs out
  Stencil C;          // cumulative weights C_j
};

template <int SR>
__global__ void __launch_bounds__(RES_MAXT, 1) k_fd_resident(const ResArgs a, const ResGeom g) {
  extern __shared__ __align__(16) float4 rsm[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int TZ = g.TZ, TX = g.TX, TXH = TX / 2, TXQ = TX / 4;
  const int RS = TXH + 4, RS2 = RS / 2;  // float4 slots per row (2 halo slots each side), per plane
  const int LV = (TZ + 8) * RS;          // float4 per (level, pair)
  float4* lv = rsm;                      // [2][P][LV]
  float4* cf = rsm + 2 * g.P * LV;       // [TZ][TXH], two planes per row
  const int tile = blockIdx.x, ntiles = g.TR * g.TC;
  const int trow = tile / g.TC, tcol = tile % g.TC;
  const int z0 = trow * TZ, x0 = tcol * TX;
  const int VR = min(TZ, a.NZ - z0);     // valid rows of this tile (>= 1)
  const bool has[4] = {trow > 0, trow + 1 < g.TR, tcol > 0, tcol + 1 < g.TC};
  const int nbr[4] = {tile - g.TC, tile + g.TC, tile - 1, tile + 1};
  const int np = a.np;
  auto sidx = [&](int r, int j) { return (r + 4) * RS + (j & 1) * RS2 + (j >> 1); };
  auto lvl = [&](int b, int p) { return lv + (size_t)(b * g.P + p) * LV; };

  // ---- load both levels (interior and halo) and the coefficients
  const int s_cur = (a.ta - 1) % 3, s_prev = (a.ta - 2 + 3) % 3;
  for (int b = 0; b < 2; ++b) {
    const int s = b == 0 ? s_cur : s_prev;
    const long long sbase = (long long)s * a.pslot * a.F;
    for (int e = tid; e < np * LV; e += nthr) {
      const int p = e / LV, k = e % LV, r = k / RS - 4, j = k % RS;
      const int z = z0 + r, x = x0 + 2 * j - 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (z >= 0 && z < a.NZ && x >= 0 && x < a.NX)
        v = __ldcg(reinterpret_cast<const float4*>(a.lev + sbase + (long long)p * a.F + a.org +
                                                   (long long)z * a.PX + x));
      lvl(b, p)[sidx(r, j)] = v;
    }
  }
  for (int e = tid; e < TZ * TXH; e += nthr) {
    const int r = e / TXH, j = e % TXH, z = z0 + r, x = x0 + 2 * j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (z < a.NZ && x < a.NX)
      v = __ldg(reinterpret_cast<const float4*>(a.coef + a.org + (long long)z * a.PX + x));
    cf[r * TXH + (j & 1) * TXQ + (j >> 1)] = v;
  }
  __syncthreads();

  float2 cz2[4], cx2[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cz2[j] = make_float2(a.C.cz[j], a.C.cz[j]);
    cx2[j] = make_float2(a.C.cx[j], a.C.cx[j]);
  }
  const int nseg = (TZ + SR - 1) / SR;
  const int nunits = np * TXQ * nseg;
  const int nN = 4 * TXH, nW = 2 * TZ, SB = 2 * nN + 2 * nW;
  bool failed = false;
  int it = 0;
  for (; it < a.nsteps; ++it) {
    const int t = a.ta + it;
    const int bc = it & 1, bn = bc ^ 1;  // current level, previous level (overwritten by the new)
    __nv_bfloat16* sl = nullptr;
    if (a.snap && t % a.decim == 0) sl = a.snap + (long long)(a.sbase + (t - a.t0) / a.decim) * a.sslot;
    for (int u = tid; u < nunits; u += nthr) {
      const int q = u % TXQ, seg = (u / TXQ) % nseg, p = u / (TXQ * nseg);
      const float4* cu = lvl(bc, p);
      float4* pv = lvl(bn, p);
      const int r0 = seg * SR;
      const int xq = x0 + 4 * q;  // padded column of the unit's first point
      // z first differences at the unit's 4 points: dz[i][m] = u(z-3+m) - u(z-4+m) for row z
      float2 dz[4][8], ul[4];
      {
        const float4 v0 = cu[sidx(r0 - 4, 2 * q + 2)], v1 = cu[sidx(r0 - 4, 2 * q + 3)];
        ul[0] = make_float2(v0.x, v0.y);
        ul[1] = make_float2(v0.z, v0.w);
        ul[2] = make_float2(v1.x, v1.y);
        ul[3] = make_float2(v1.z, v1.w);
      }
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        const float4 v0 = cu[sidx(r0 - 4 + k, 2 * q + 2)], v1 = cu[sidx(r0 - 4 + k, 2 * q + 3)];
        const float2 nv[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                              make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          dz[i][k] = rsub2(nv[i], ul[i]);
          ul[i] = nv[i];
        }
      }
#pragma unroll
      for (int ii = 0; ii < SR; ++ii) {
        const int r = r0 + ii;
        if (r >= TZ) break;
        {
          const float4 v0 = cu[sidx(r + 4, 2 * q + 2)], v1 = cu[sidx(r + 4, 2 * q + 3)];
          const float2 nv[4] = {make_float2(v0.x, v0.y), make_float2(v0.z, v0.w),
                                make_float2(v1.x, v1.y), make_float2(v1.z, v1.w)};
#pragma unroll
          for (int i = 0; i < 4; ++i) {
#pragma unroll
            for (int m = 0; m < 7; ++m) dz[i][m] = dz[i][m + 1];
            dz[i][7] = rsub2(nv[i], ul[i]);
            ul[i] = nv[i];
          }
        }
        // u^n at row r, points 4q - 4 .. 4q + 7 (both receivers of the pair)
        float2 w[12];
#pragma unroll
        for (int s = 0; s < 6; ++s) {
          const float4 A = cu[sidx(r, 2 * q + s)];
          w[2 * s] = make_float2(A.x, A.y);
          w[2 * s + 1] = make_float2(A.z, A.w);
        }
        float2 e[11];
#pragma unroll
        for (int m = 0; m < 11; ++m) e[m] = rsub2(w[m + 1], w[m]);
        const float4 o01 = pv[sidx(r, 2 * q + 2)], o23 = pv[sidx(r, 2 * q + 3)];
        const float4 c01 = cf[r * TXH + q], c23 = cf[r * TXH + TXQ + q];
        const float2 o[4] = {make_float2(o01.x, o01.y), make_float2(o01.z, o01.w),
                             make_float2(o23.x, o23.y), make_float2(o23.z, o23.w)};
        const float2 c1[4] = {make_float2(c01.x, c01.x), make_float2(c01.z, c01.z),
                              make_float2(c23.x, c23.x), make_float2(c23.z, c23.z)};
        const float2 c3[4] = {make_float2(c01.y, c01.y), make_float2(c01.w, c01.w),
                              make_float2(c23.y, c23.y), make_float2(c23.w, c23.w)};
        float2 v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float2 l = rlap2(dz[i], e + i, cz2, cx2);
          // u^{n+1} = c3 L u + c1 (u - u^{n-1}) + u^{n-1}
          v[i] = __ffma2_rn(c3[i], l, __ffma2_rn(c1[i], rsub2(w[i + 4], o[i]), o[i]));
          if (xq + i >= a.NX) v[i] = make_float2(0.f, 0.f);
        }
        if (r < VR && xq < a.NX) {
          pv[sidx(r, 2 * q + 2)] = make_float4(v[0].x, v[0].y, v[1].x, v[1].y);
          pv[sidx(r, 2 * q + 3)] = make_float4(v[2].x, v[2].y, v[3].x, v[3].y);
          if (sl) {
            unsigned ha0, la0, ha1, la1, hb0, lb0, hb1, lb1;
            rsplit(v[0].x, v[1].x, ha0, la0);
            rsplit(v[2].x, v[3].x, ha1, la1);
            rsplit(v[0].y, v[1].y, hb0, lb0);
            rsplit(v[2].y, v[3].y, hb1, lb1);
            __nv_bfloat16* sp = sl + (long long)(2 * p) * a.srec + (long long)(z0 + r) * a.PX + xq;
            __stcs(reinterpret_cast<uint2*>(sp), make_uint2(ha0, ha1));
            __stcs(reinterpret_cast<uint2*>(sp + a.splane), make_uint2(la0, la1));
            __stcs(reinterpret_cast<uint2*>(sp + a.srec), make_uint2(hb0, hb1));
            __stcs(reinterpret_cast<uint2*>(sp + a.srec + a.splane), make_uint2(lb0, lb1));
          }
        }
      }
    }
    __syncthreads();  // the new level is complete in shared memory
    // ---- publish the new level's boundary strips, then this block's step count
    float4* xme = a.xbuf + ((size_t)(it & 1) * ntiles + tile) * g.P * SB;
    for (int e = tid; e < np * SB; e += nthr) {
      const int p = e / SB, k = e % SB;
      int r, j;
      if (k < nN) {
        if (!has[0]) continue;
        r = k / TXH;
        j = 2 + k % TXH;
      } else if (k < 2 * nN) {
        if (!has[1]) continue;
        r = TZ - 4 + (k - nN) / TXH;
        j = 2 + (k - nN) % TXH;
      } else if (k < 2 * nN + nW) {
        if (!has[2]) continue;
        r = (k - 2 * nN) >> 1;
        j = 2 + ((k - 2 * nN) & 1);
      } else {
        if (!has[3]) continue;
        r = (k - 2 * nN - nW) >> 1;
        j = RS - 4 + ((k - 2 * nN - nW) & 1);
      }
      __stcg(xme + (size_t)p * SB + k, lvl(bn, p)[sidx(r, j)]);
    }
    __syncthreads();
    if (tid == 0) {
      __threadfence();
      st_release(a.flags + tile, it + 1);
    }
    // ---- wait for the neighbours' strips of this step (bounded; an abort ends every wait)
    bool ok = true;
    if (tid < 4 && has[tid]) {
      const int* f = a.flags + nbr[tid];
      const unsigned long long tw0 = tc::globaltimer_ns();
      long long polls = 0;
      while (ld_acquire(f) < it + 1) {
        if (ld_relaxed(a.abort_flag)) {
          ok = false;
          break;
        }
        if ((++polls & 15) == 0 && tc::globaltimer_ns() - tw0 > tc::kWaitNs) {
          ok = false;
          atomicExch(a.err, 1);
          atomicExch(a.abort_flag, 1);
          break;
        }
      }
    }
    if (it == 0 && a.expire && tile == 0 && tid == 0) {
      // test hook: wait for a step count that no block ever publishes, for a short time
      const unsigned long long tw0 = tc::globaltimer_ns();
      while (ld_acquire(a.flags + tile) < INT_MAX) {
        if (tc::globaltimer_ns() - tw0 > tc::kExpireNs) {
          ok = false;
          atomicExch(a.err, 1);
          atomicExch(a.abort_flag, 1);
          break;
        }
      }
    }
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    if (it + 1 == a.nsteps) break;  // the last level needs no halo
    // ---- the neighbours' strips into the new level's halo
    const float4* xb = a.xbuf + (size_t)(it & 1) * ntiles * g.P * SB;
    for (int e = tid; e < np * SB; e += nthr) {
      const int p = e / SB, k = e % SB;
      int r, j;
      const float4* src;
      if (k < nN) {  // rows -4 .. -1 <- the upper tile's last four rows
        if (!has[0]) continue;
        r = -4 + k / TXH;
        j = 2 + k % TXH;
        src = xb + ((size_t)nbr[0] * g.P + p) * SB + nN + k;
      } else if (k < 2 * nN) {  // rows TZ .. TZ + 3 <- the lower tile's first four rows
        if (!has[1]) continue;
        const int kk = k - nN;
        r = TZ + kk / TXH;
        j = 2 + kk % TXH;
        src = xb + ((size_t)nbr[1] * g.P + p) * SB + kk;
      } else if (k < 2 * nN + nW) {  // columns -4 .. -1 <- the left tile's last four columns
        if (!has[2]) continue;
        const int kk = k - 2 * nN;
        r = kk >> 1;
        j = kk & 1;
        src = xb + ((size_t)nbr[2] * g.P + p) * SB + 2 * nN + nW + kk;
      } else {  // columns TX .. TX + 3 <- the right tile's first four columns
        if (!has[3]) continue;
        const int kk = k - 2 * nN - nW;
        r = kk >> 1;
        j = RS - 2 + (kk & 1);
        src = xb + ((size_t)nbr[3] * g.P + p) * SB + 2 * nN + kk;
      }
      lvl(bn, p)[sidx(r, j)] = __ldcg(src);
    }
    __syncthreads();
  }
  if (failed) return;
  // ---- the last two levels back to their state slots (valid interior points)
  const int t1 = a.ta + a.nsteps;
  for (int b = 0; b < 2; ++b) {
    const int buf = b == 0 ? (a.nsteps & 1) : ((a.nsteps + 1) & 1);
    const int s = b == 0 ? (t1 - 1) % 3 : (t1 - 2) % 3;
    const long long sbase = (long long)s * a.pslot * a.F;
    for (int e = tid; e < np * VR * TXH; e += nthr) {
      const int p = e / (VR * TXH), k = e % (VR * TXH), r = k / TXH, j = 2 + k % TXH;
      const int z = z0 + r, x = x0 + 2 * j - 4;
      if (x < a.NX)
        __stcg(reinterpret_cast<float4*>(a.lev + sbase + (long long)p * a.F + a.org +
                                         (long long)z * a.PX + x),
               lvl(buf, p)[sidx(r, j)]);
    }
  }
}

int res_threads(const ResGeom& g, int sr, int np) {
  const int units = np * (g.TX / 4) * ((g.TZ + sr - 1) / sr);
  return std::max(32, std::min(RES_MAXT, (units + 31) / 32 * 32));
}

}  // namespace

// Shared memory of a tile: both levels of P pairs with their halos, and the coefficients.
static size_t res_smem(int TZ, int TX, int P) {
  return sizeof(float4) * ((size_t)2 * P * (TZ + 8) * (TX / 2 + 4) + (size_t)TZ * (TX / 2));
}

bool fd_resident_plan(const Layout& L, int want_pairs, ResGeom* out) {
  int dev = 0, sms = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return false;
  ResGeom best{};
  long long best_area = LLONG_MAX;
  for (int tr = 1; tr <= std::min(sms, L.NZ); ++tr) {
    const int TZ = (L.NZ + tr - 1) / tr;
    const int TR = (L.NZ + TZ - 1) / TZ;
    const int tcmax = sms / TR;
    if (tcmax < 1) break;
    const int TX = ((L.NX + tcmax - 1) / tcmax + 3) / 4 * 4;
    const int TC = (L.NX + TX - 1) / TX;
    if (TR * TC > sms || TZ < 4 || TX < 4) continue;
    int P = std::min(want_pairs, 8);
    while (P >= 1 && res_smem(TZ, TX, P) > (size_t)optin) --P;
    if (P < 1) continue;
    const long long area = (long long)(TZ + 8) * (TX + 8);  // with the halo: shared-memory traffic per step
    // most pairs first (fewer batches, fewer exchanges per receiver), then the smallest tile
    if (P > best.P || (P == best.P && area < best_area)) {
      best = ResGeom{TR, TC, TZ, TX, P, res_smem(TZ, TX, P)};
      best_area = area;
    }
  }
  if (best.P < 1) return false;
  *out = best;
  return true;
}

size_t fd_resident_xbuf_float4(const ResGeom& g) {
  return (size_t)2 * g.TR * g.TC * g.P * (8 * (g.TX / 2) + 4 * g.TZ);
}

static const int kSR[] = {6, 8, 11, 16};

int fd_resident_sr_default() { return 8; }

bool fd_resident_sr_valid(int sr) {
  for (int v : kSR)
    if (v == sr) return true;
  return false;
}

cudaError_t fd_resident_prepare(const ResGeom& g, int sr, int np) {
  cudaError_t e;
#define EGH_RES_ATTR(S)                                                                          \
  if ((e = cudaFuncSetAttribute(k_fd_resident<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,   \
                                (int)g.smem)))                                                   \
    return e;
  EGH_RES_ATTR(6)
  EGH_RES_ATTR(8)
  EGH_RES_ATTR(11)
  EGH_RES_ATTR(16)
#undef EGH_RES_ATTR
  // every block must be resident at once (one per SM) for the neighbour waits
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) || (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)))
    return e;
  const int thr = res_threads(g, sr, np);
  switch (sr) {
    case 6: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fd_resident<6>, thr, g.smem); break;
    case 8: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fd_resident<8>, thr, g.smem); break;
    case 11: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fd_resident<11>, thr, g.smem); break;
    case 16: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_fd_resident<16>, thr, g.smem); break;
    default: return cudaErrorInvalidValue;
  }
  if (e) return e;
  if ((long long)occ * sms < (long long)g.TR * g.TC) return cudaErrorCooperativeLaunchTooLarge;
  return cudaSuccess;
}

cudaError_t launch_fd_resident(const ResGeom& g, int sr, float2* lev, int pslot, const Layout& L,
                               const float2* coef, const Stencil& S, int np, int ta, int nsteps,
                               int t0, int decim, int sbase, __nv_bfloat16* snap, long long sslot,
                               long long splane, long long srec, float4* xbuf, int* flags,
                               int* err, int expire, cudaStream_t st) {
  if (np < 1 || np > g.P || nsteps < 1 || ta < 2 || decim < 1 || g.TX % 4 != 0)
    return cudaErrorInvalidValue;
  ResArgs a{};
  a.lev = lev;
  a.F = L.F;
  a.pslot = pslot;
  a.org = L.org;
  a.NZ = L.NZ;
  a.NX = L.NX;
  a.PX = L.PX;
  a.coef = coef;
  a.np = np;
  a.ta = ta;
  a.nsteps = nsteps;
  a.t0 = t0;
  a.decim = decim;
  a.sbase = sbase;
  a.snap = snap;
  a.sslot = sslot;
  a.splane = splane;
  a.srec = srec;
  a.xbuf = xbuf;
  a.flags = flags;
  a.abort_flag = flags + g.TR * g.TC;
  a.err = err;
  a.expire = expire;
  // cumulative weights C_j = sum_{k>=j} c_k of the first-difference form (as fd.cu)
  float az = 0.f, ax = 0.f;
  for (int k = 3; k >= 0; --k) {
    az += S.cz[k];
    ax += S.cx[k];
    a.C.cz[k] = az;
    a.C.cx[k] = ax;
  }
  cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int) * (g.TR * g.TC + 1), st);
  if (e != cudaSuccess) return e;
  ResGeom gg = g;
  void* args[] = {&a, &gg};
  const dim3 grid(g.TR * g.TC), block(res_threads(g, sr, np));
  count_launches(1);
  switch (sr) {
    case 6: return cudaLaunchCooperativeKernel((void*)k_fd_resident<6>, grid, block, args, g.smem, st);
    case 8: return cudaLaunchCooperativeKernel((void*)k_fd_resident<8>, grid, block, args, g.smem, st);
    case 11: return cudaLaunchCooperativeKernel((void*)k_fd_resident<11>, grid, block, args, g.smem, st);
    case 16: return cudaLaunchCooperativeKernel((void*)k_fd_resident<16>, grid, block, args, g.smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace egh
