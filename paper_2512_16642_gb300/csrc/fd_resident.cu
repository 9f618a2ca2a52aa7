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
// Work inside a block: the batch's pairs are split into NG groups; each group is a set of warps
// with its own named barrier and its own step counters, so that while one group waits for its
// neighbours' strips the other computes.  A unit is (receiver pair, 2 adjacent columns, a segment
// of SR rows): its thread marches down the segment with the z first differences in registers, as
// fd.cu does, and reads the x neighbours from shared memory (one float4 = both receivers of the
// pair at 2 points, adjacent threads on adjacent words).
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

constexpr int RES_MAXT = 640;  // threads per block at most
// threads per block at most for SR rows per segment: short segments (more units) take more
// threads at fewer registers; long segments keep their window in registers at fewer threads
__host__ __device__ constexpr int res_maxt(int sr) { return sr <= 8 ? 640 : 448; }
constexpr int RES_E = 4;  // exchange elements of a pair per thread at most

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
// named barrier `id` over `n` threads (whole warps)
__device__ __forceinline__ void gbar(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// the same with an OR of a predicate over the participating threads
__device__ __forceinline__ bool gbar_or(int id, int n, bool pred) {
  unsigned r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, %2, %3, p;\n"
      " selp.u32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((unsigned)pred), "r"(id), "r"(n)
      : "memory");
  return r != 0;
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
  int* flags;         // [NG][tiles] steps completed in this launch, then the abort flag (zeroed
                      // before the launch)
  int* err;           // the context's error flag
  int expire;         // test hook: block 0's first wait runs out
  int GT;             // threads per group (whole warps)
  Stencil C;          // cumulative weights C_j
};

template <int SR>
__global__ void __launch_bounds__(res_maxt(SR), 1) k_fd_resident(const ResArgs a, const ResGeom g) {
  extern __shared__ __align__(16) float4 rsm[];
  const int tid = threadIdx.x, nthr = blockDim.x;
  const int TZ = g.TZ, TX = g.TX, TXH = TX / 2;
  const int RS = TXH + 4;                // float4 slots per row (2 halo slots each side)
  const int LV = (TZ + 8) * RS;          // float4 per (level, pair)
  float4* lv = rsm;                      // [2][P][LV]
  float4* cf = rsm + 2 * g.P * LV;       // [TZ][TXH]
  const int tile = blockIdx.x, ntiles = g.TR * g.TC;
  const int trow = tile / g.TC, tcol = tile % g.TC;
  const int z0 = trow * TZ, x0 = tcol * TX;
  const int VR = min(TZ, a.NZ - z0);     // valid rows of this tile (>= 1)
  const bool has[4] = {trow > 0, trow + 1 < g.TR, tcol > 0, tcol + 1 < g.TC};
  const int nbr[4] = {tile - g.TC, tile + g.TC, tile - 1, tile + 1};
  const int np = a.np;
  auto lvl = [&](int b, int p) { return lv + (size_t)(b * g.P + p) * LV; };
  auto sidx = [&](int r, int j) { return (r + 4) * RS + j; };

  // ---- load both levels (interior and halo) and the coefficients (whole block)
  const int s_cur = (a.ta - 1) % 3, s_prev = (a.ta - 2 + 3) % 3;
  for (int b = 0; b < 2; ++b) {
    const int s = b == 0 ? s_cur : s_prev;
    const long long sb = (long long)s * a.pslot * a.F;
    for (int e = tid; e < np * LV; e += nthr) {
      const int p = e / LV, k = e % LV, r = k / RS - 4, j = k % RS;
      const int z = z0 + r, x = x0 + 2 * j - 4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (z >= 0 && z < a.NZ && x >= 0 && x < a.NX)
        v = __ldcg(reinterpret_cast<const float4*>(a.lev + sb + (long long)p * a.F + a.org +
                                                   (long long)z * a.PX + x));
      lvl(b, p)[k] = v;
    }
  }
  for (int e = tid; e < TZ * TXH; e += nthr) {
    const int r = e / TXH, j = e % TXH, z = z0 + r, x = x0 + 2 * j;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (z < a.NZ && x < a.NX)
      v = __ldg(reinterpret_cast<const float4*>(a.coef + a.org + (long long)z * a.PX + x));
    cf[e] = v;
  }
  __syncthreads();

  // ---- this thread's group: pairs [p0, p1), local thread lt of GT, barrier id 1 + gi
  const int GT = a.GT, gi = tid / GT, lt = tid % GT;
  const int NG = nthr / GT, PG = (g.P + NG - 1) / NG;
  const int p0 = min(np, gi * PG), p1 = min(np, p0 + PG);
  const int bid = 1 + gi;
  int* gflags = a.flags + gi * ntiles;
  int* abort_flag = a.flags + NG * ntiles;
  // strip elements k = lt + i GT (i < RES_E) of a pair's SB-float4 exchange block: N = rows 0..3,
  // S = rows TZ-4..TZ-1 (4 x TXH each), W = columns 0..3, E = columns TX-4..TX-1 (TZ x 2 each).
  // Publishing copies the new level's boundary element to the block; filling copies the matching
  // neighbour element into the halo.  Packed: pub slot | halo slot << 16, and neighbour offset |
  // side << 16 | valid << 18.
  const int nN = 4 * TXH, nW = 2 * TZ, SB = 2 * nN + 2 * nW;
  int ent_s[RES_E], ent_n[RES_E];
#pragma unroll
  for (int i = 0; i < RES_E; ++i) {
    const int k = lt + i * GT;
    int pub = 0, halo = 0, src = 0, side = 0, valid = 0;
    if (k < SB) {
      if (k < nN) {  // N: rows 0..3 <-> the upper tile fills my rows -4..-1 from its S
        side = 0;
        pub = sidx(k / TXH, 2 + k % TXH);
        halo = sidx(-4 + k / TXH, 2 + k % TXH);
        src = nN + k;
      } else if (k < 2 * nN) {  // S: rows TZ-4..TZ-1 <-> my rows TZ..TZ+3 from the lower N
        const int kk = k - nN;
        side = 1;
        pub = sidx(TZ - 4 + kk / TXH, 2 + kk % TXH);
        halo = sidx(TZ + kk / TXH, 2 + kk % TXH);
        src = kk;
      } else if (k < 2 * nN + nW) {  // W: columns 0..3 <-> my columns -4..-1 from the left E
        const int kk = k - 2 * nN;
        side = 2;
        pub = sidx(kk >> 1, 2 + (kk & 1));
        halo = sidx(kk >> 1, kk & 1);
        src = k + nW;
      } else {  // E: columns TX-4..TX-1 <-> my columns TX..TX+3 from the right W
        const int kk = k - 2 * nN - nW;
        side = 3;
        pub = sidx(kk >> 1, RS - 4 + (kk & 1));
        halo = sidx(kk >> 1, RS - 2 + (kk & 1));
        src = k - nW;
      }
      valid = has[side] ? 1 : 0;
    }
    ent_s[i] = pub | (halo << 16);
    ent_n[i] = src | (side << 16) | (valid << 18);
  }

  float2 cz2[4], cx2[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cz2[j] = make_float2(a.C.cz[j], a.C.cz[j]);
    cx2[j] = make_float2(a.C.cx[j], a.C.cx[j]);
  }
  const int nseg = (TZ + SR - 1) / SR;
  const int nunits = (p1 - p0) * TXH * nseg;
  bool failed = false;
  for (int it = 0; it < a.nsteps; ++it) {
    const int t = a.ta + it;
    const int bc = it & 1, bn = bc ^ 1;  // current level, previous level (overwritten by the new)
    __nv_bfloat16* sl = nullptr;
    if (a.snap && t % a.decim == 0) sl = a.snap + (long long)(a.sbase + (t - a.t0) / a.decim) * a.sslot;
    for (int u = lt; u < nunits; u += GT) {
      const int q = u % TXH, seg = (u / TXH) % nseg, p = p0 + u / (TXH * nseg);
      const float4* cu = lvl(bc, p) + q;  // slot q + 2 is this unit's centre
      float4* pv = lvl(bn, p) + q + 2;
      const float4* cq = cf + q;
      const int r0 = seg * SR;
      const int x = x0 + 2 * q;  // padded column of the unit's first point
      const bool ok0 = x < a.NX, ok1 = x + 1 < a.NX;
      // z first differences: dz[pt][m] = u(z-3+m) - u(z-4+m) at the current row z
      float2 dz[2][8], ul[2];
      {
        const float4 v = cu[sidx(r0 - 4, 2)];
        ul[0] = make_float2(v.x, v.y);
        ul[1] = make_float2(v.z, v.w);
      }
#pragma unroll
      for (int k = 1; k < 8; ++k) {
        const float4 v = cu[sidx(r0 - 4 + k, 2)];
        const float2 nv[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
        for (int i = 0; i < 2; ++i) {
          dz[i][k] = rsub2(nv[i], ul[i]);
          ul[i] = nv[i];
        }
      }
#pragma unroll
      for (int ii = 0; ii < SR; ++ii) {
        const int r = r0 + ii;
        if (r >= TZ) break;
        {
          const float4 v = cu[sidx(r + 4, 2)];
          const float2 nv[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
          for (int i = 0; i < 2; ++i) {
#pragma unroll
            for (int m = 0; m < 7; ++m) dz[i][m] = dz[i][m + 1];
            dz[i][7] = rsub2(nv[i], ul[i]);
            ul[i] = nv[i];
          }
        }
        // u^n at row r, points x - 4 .. x + 5 (both receivers of the pair)
        const float4* xr = cu + sidx(r, 0);
        const float4 A0 = xr[0], A1 = xr[1], A2 = xr[2], A3 = xr[3], A4 = xr[4];
        const float2 w[10] = {make_float2(A0.x, A0.y), make_float2(A0.z, A0.w), make_float2(A1.x, A1.y),
                              make_float2(A1.z, A1.w), make_float2(A2.x, A2.y), make_float2(A2.z, A2.w),
                              make_float2(A3.x, A3.y), make_float2(A3.z, A3.w), make_float2(A4.x, A4.y),
                              make_float2(A4.z, A4.w)};
        float2 e[9];
#pragma unroll
        for (int m = 0; m < 9; ++m) e[m] = rsub2(w[m + 1], w[m]);
        const float4 uo = pv[sidx(r, 0)], cc = cq[r * TXH];
        const float2 l0 = rlap2(dz[0], e, cz2, cx2), l1 = rlap2(dz[1], e + 1, cz2, cx2);
        // u^{n+1} = c3 L u + c1 (u - u^{n-1}) + u^{n-1}
        const float2 o0 = make_float2(uo.x, uo.y), o1 = make_float2(uo.z, uo.w);
        const float2 v0 = __ffma2_rn(make_float2(cc.y, cc.y), l0,
                                     __ffma2_rn(make_float2(cc.x, cc.x), rsub2(w[4], o0), o0));
        float2 v1 = __ffma2_rn(make_float2(cc.w, cc.w), l1,
                               __ffma2_rn(make_float2(cc.z, cc.z), rsub2(w[5], o1), o1));
        if (!ok1) v1 = make_float2(0.f, 0.f);
        if (r < VR && ok0) {
          pv[sidx(r, 0)] = make_float4(v0.x, v0.y, v1.x, v1.y);
          if (sl) {
            unsigned ha, la, hb, lb;
            rsplit(v0.x, v1.x, ha, la);
            rsplit(v0.y, v1.y, hb, lb);
            __nv_bfloat16* sp = sl + (long long)(2 * p) * a.srec + (long long)(z0 + r) * a.PX + x;
            __stcs(reinterpret_cast<unsigned*>(sp), ha);
            __stcs(reinterpret_cast<unsigned*>(sp + a.splane), la);
            __stcs(reinterpret_cast<unsigned*>(sp + a.srec), hb);
            __stcs(reinterpret_cast<unsigned*>(sp + a.srec + a.splane), lb);
          }
        }
      }
    }
    gbar(bid, GT);  // the group's new level is complete in shared memory
    // ---- publish the new level's boundary strips, then the group's step count
    float4* xme = a.xbuf + ((size_t)(it & 1) * ntiles + tile) * g.P * SB;
#pragma unroll
    for (int i = 0; i < RES_E; ++i)
      if ((ent_n[i] >> 18) & 1)
        for (int p = p0; p < p1; ++p)
          __stcg(xme + (size_t)p * SB + lt + i * GT, lvl(bn, p)[ent_s[i] & 0xffff]);
    gbar(bid, GT);
    if (lt == 0) {
      __threadfence();
      st_release(gflags + tile, it + 1);
    }
    // ---- wait for the neighbours' strips of this step (bounded; an abort ends every wait)
    bool ok = true;
    if (lt < 4 && has[lt] && p1 > p0) {
      const int* f = gflags + nbr[lt];
      const unsigned long long tw0 = tc::globaltimer_ns();
      long long polls = 0;
      while (ld_acquire(f) < it + 1) {
        if (ld_relaxed(abort_flag)) {
          ok = false;
          break;
        }
        if ((++polls & 15) == 0 && tc::globaltimer_ns() - tw0 > tc::kWaitNs) {
          ok = false;
          atomicExch(a.err, 1);
          atomicExch(abort_flag, 1);
          break;
        }
      }
    }
    if (it == 0 && a.expire && tile == 0 && tid == 0) {
      // test hook: wait for a step count that no block ever publishes, for a short time
      const unsigned long long tw0 = tc::globaltimer_ns();
      while (ld_acquire(gflags + tile) < INT_MAX) {
        if (tc::globaltimer_ns() - tw0 > tc::kExpireNs) {
          ok = false;
          atomicExch(a.err, 1);
          atomicExch(abort_flag, 1);
          break;
        }
      }
    }
    if (gbar_or(bid, GT, !ok)) {
      failed = true;
      break;
    }
    if (it + 1 == a.nsteps) break;  // the last level needs no halo
    // ---- the neighbours' strips into the new level's halo
    const float4* xb = a.xbuf + (size_t)(it & 1) * ntiles * g.P * SB;
#pragma unroll
    for (int i = 0; i < RES_E; ++i)
      if ((ent_n[i] >> 18) & 1) {
        const float4* src = xb + (size_t)nbr[(ent_n[i] >> 16) & 3] * g.P * SB + (ent_n[i] & 0xffff);
        for (int p = p0; p < p1; ++p) lvl(bn, p)[ent_s[i] >> 16] = __ldcg(src + (size_t)p * SB);
      }
    gbar(bid, GT);
  }
  // every group has left its loop (a failed group may leave early; the others then see its abort)
  if (__syncthreads_or(failed)) return;
  // ---- the last two levels back to their state slots (valid interior points)
  const int t1 = a.ta + a.nsteps;
  for (int b = 0; b < 2; ++b) {
    const int buf = b == 0 ? (a.nsteps & 1) : ((a.nsteps + 1) & 1);
    const int s = b == 0 ? (t1 - 1) % 3 : (t1 - 2) % 3;
    const long long sb = (long long)s * a.pslot * a.F;
    for (int e = tid; e < np * VR * TXH; e += nthr) {
      const int p = e / (VR * TXH), k = e % (VR * TXH), r = k / TXH, j = 2 + k % TXH;
      const int z = z0 + r, x = x0 + 2 * j - 4;
      if (x < a.NX)
        __stcg(reinterpret_cast<float4*>(a.lev + sb + (long long)p * a.F + a.org +
                                         (long long)z * a.PX + x),
               lvl(buf, p)[sidx(r, j)]);
    }
  }
}

// Pair groups per block (two when there are two pairs or more, so that one group computes while
// the other exchanges) and threads per group: one per unit, enough that no thread handles more
// than RES_E exchange elements of a pair, whole warps.
int res_groups(const ResGeom& g) { return g.P >= 2 ? 2 : 1; }
int res_group_threads(const ResGeom& g, int sr) {
  const int NG = res_groups(g), PG = (g.P + NG - 1) / NG;
  const int units = PG * (g.TX / 2) * ((g.TZ + sr - 1) / sr);
  const int SB = 8 * (g.TX / 2) + 4 * g.TZ;
  const int gt = std::max((units + 31) / 32, (SB + 32 * RES_E - 1) / (32 * RES_E)) * 32;
  return std::min(gt, res_maxt(sr) / NG / 32 * 32);
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
    // no thread of a group takes more than RES_E exchange elements of a pair
    if (8 * (TX / 2) + 4 * TZ > RES_E * (res_maxt(16) / 2 / 32 * 32)) continue;
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

size_t fd_resident_flags(const ResGeom& g) { return (size_t)res_groups(g) * g.TR * g.TC + 1; }

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
  const int thr = res_groups(g) * res_group_threads(g, sr);
  (void)np;
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
  a.err = err;
  a.expire = expire;
  a.GT = res_group_threads(g, sr);
  // cumulative weights C_j = sum_{k>=j} c_k of the first-difference form (as fd.cu)
  float az = 0.f, ax = 0.f;
  for (int k = 3; k >= 0; --k) {
    az += S.cz[k];
    ax += S.cx[k];
    a.C.cz[k] = az;
    a.C.cx[k] = ax;
  }
  cudaError_t e =
      cudaMemsetAsync(flags, 0, sizeof(int) * ((size_t)res_groups(g) * g.TR * g.TC + 1), st);
  if (e != cudaSuccess) return e;
  ResGeom gg = g;
  void* args[] = {&a, &gg};
  const dim3 grid(g.TR * g.TC), block(res_groups(g) * a.GT);
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
