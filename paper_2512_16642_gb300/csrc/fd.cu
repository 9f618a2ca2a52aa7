// Time-domain finite differences for the receiver-side Green functions and their on-the-fly
// transform at the Nf frequencies (Section "Direct Hessian-inverse computation": one wave-equation
// solve per receiver with a Dirac source at the receiver; eq. wave_eq).
//
// Scheme (the paper does not give one): second-order leapfrog, eighth-order Laplacian, damping
// written symmetrically so that reciprocity holds,
//     u^{n+1} = c1 (u^n - u^{n-1}) + u^{n-1} + c3 L u^n,   c1 = 2/(1+a), c3 = dt^2 v^2/(1+a),
// a = eta dt / 2 (from (1+a) u^{n+1} = 2 u^n - (1-a) u^{n-1} + dt^2 v^2 L u^n, since
// (1-a)/(1+a) = c1 - 1).
//
// Receivers are propagated in pairs: a level of a pair stores float2 (receiver 2i, receiver 2i+1)
// per grid point, so every load, store and arithmetic instruction of the step serves two
// receivers (packed FP32x2 arithmetic of sm_100+).
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <cstring>
#include <vector>

#include "egh_internal.cuh"
#include "tc.cuh"

namespace egh {

// ---------------------------------------------------------------------------------------------
// Velocity check: d_out[0] = max velocity, d_out[1] = count of non-positive / non-finite values.
// ---------------------------------------------------------------------------------------------
__global__ void k_check_velocity(const float* __restrict__ vel, long long n, float* out) {
  float vmax = 0.f;
  int bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = vel[i];
    if (!(v > 0.f) || !isfinite(v)) {
      ++bad;
    } else {
      vmax = fmaxf(vmax, v);
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    vmax = fmaxf(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
    bad += __shfl_xor_sync(0xffffffffu, bad, o);
  }
  if ((threadIdx.x & 31) == 0) {
    // positive floats order like their bit patterns
    atomicMax(reinterpret_cast<int*>(out), __float_as_int(vmax));
    if (bad) atomicAdd(out + 1, (float)bad);
  }
}

cudaError_t launch_check_velocity(const float* vel, long long n, float* d_out, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_out, 0, 2 * sizeof(float), st);
  if (e != cudaSuccess) return e;
  long long blocks = (n + 255) / 256;
  if (blocks > 1216) blocks = 1216;
  count_launches(1);
  k_check_velocity<<<(int)blocks, 256, 0, st>>>(vel, n, d_out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Coefficients (c1, c3) on the padded, pitched grid.  Velocity is extended into the sponge by
// edge replication; eta = eta0 (d/L)^2 per axis, eta0 = 1.5 vmax ln(1/R) / L.
// ---------------------------------------------------------------------------------------------
__device__ inline double sponge_profile(int i, int N, int ns, double h, double eta0) {
  int d = 0;
  if (i < ns) d = ns - i;
  if (i > N - 1 - ns) d = max(d, i - (N - 1 - ns));
  const double L = ns * h;
  const double r = d * h / L;
  return eta0 * r * r;
}

__global__ void k_build_coef(const float* __restrict__ vel, Layout L, double dz, double dx,
                             double dt, double R, const float* __restrict__ d_vmax,
                             float2* __restrict__ coef) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (x >= L.PX || z >= L.NZ) return;
  const long long p = L.org + (long long)z * L.PX + x;
  if (x >= L.NX) {
    coef[p] = make_float2(0.f, 0.f);
    return;
  }
  const int iz = min(max(z - L.ns, 0), L.nz - 1);
  const int ix = min(max(x - L.ns, 0), L.nx - 1);
  const double v = vel[(long long)iz * L.nx + ix];
  double eta = 0.0;
  if (L.ns > 0) {
    const double vmax = d_vmax[0];
    const double lr = log(1.0 / R);
    eta = sponge_profile(z, L.NZ, L.ns, dz, 1.5 * vmax * lr / (L.ns * dz)) +
          sponge_profile(x, L.NX, L.ns, dx, 1.5 * vmax * lr / (L.ns * dx));
  }
  const double a = 0.5 * eta * dt;
  coef[p] = make_float2((float)(2.0 / (1.0 + a)), (float)(dt * dt * v * v / (1.0 + a)));
}

cudaError_t launch_build_coef(const float* vel, const Layout& L, double dz, double dx, double dt,
                              double R, const float* d_vmax, float2* coef, cudaStream_t st) {
  dim3 grid((L.PX + 127) / 128, L.NZ);
  count_launches(1);
  k_build_coef<<<grid, 128, 0, st>>>(vel, L, dz, dx, dt, R, d_vmax, coef);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// One leapfrog step for a batch of receiver pairs.  A warp owns 64 columns of one pair, two
// adjacent points per lane (one float4 = both receivers at both points), and marches down TZ rows
// (fully unrolled, so the z-window rotates through registers).  The u^n rows stream through a
// per-warp ring of FD_RING shared-memory rows (64 points + 4 halo points on each side) filled by
// cp.async FD_D rows ahead of use; the same ring rows give the x-neighbours (five 16-byte loads
// per lane).  u^{n-1} and the coefficients are prefetched into registers FD_P rows ahead.  Reads
// of guard rows and padding columns return the zero boundary, so loads need no bounds test.
//
// The Laplacian is taken in first differences: with D_j = u_j - u_{j-1} along an axis,
//   sum_k c_k (u_{+k} + u_{-k} - 2u) = sum_{j=1..4} C_j (D_{+j} - D_{1-j}),  C_j = sum_{k>=j} c_k,
// so every rounding is relative to neighbour differences (the large cancelling terms of
// c_0 u + sum_k c_k (u_{+k} + u_{-k}) never form) and each first difference is formed once.
//
// The new level goes to its state slot and, when `so.lvl` is set, its bf16 split u = hi + lo
// (hi = bf16(u), lo = bf16(u - hi); about 2^-17 relative) goes to the snapshot ring the
// transform reads.
// ---------------------------------------------------------------------------------------------
#ifndef EGH_FD_P
#define EGH_FD_P 2
#endif
#ifndef EGH_FD_MINB
#define EGH_FD_MINB 1
#endif
constexpr int FD_RING = 12;     // ring rows per warp (indices are compile-time: any count)
constexpr int FD_D = 7;         // u^n rows in flight ahead of the window's leading row
constexpr int FD_P = EGH_FD_P;  // u^{n-1} / coefficient rows prefetched ahead
static_assert(FD_D + 5 <= FD_RING && FD_D + 8 >= FD_RING, "ring rows must cover the prefetch distance");

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}

__device__ __forceinline__ unsigned bf2_bits(__nv_bfloat162 v) {
  return *reinterpret_cast<unsigned*>(&v);
}

// hi/lo bf16 split of two values of one receiver at adjacent points, packed (point x, point x+1)
__device__ __forceinline__ void split_bf16(float a, float b, unsigned& hi, unsigned& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const float2 r = sub2(make_float2(a, b), hf);
  hi = bf2_bits(h);
  lo = bf2_bits(__floats2bfloat162_rn(r.x, r.y));
}

__device__ __forceinline__ void cp_async16(unsigned dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// The first-difference Laplacian of both receivers of a pair at once (float2 = receivers (a, b)),
// in packed FP32x2 instructions: the kernel is bound by instruction issue, and one packed
// instruction does the work of two scalar ones (same roundings).  C holds the cumulative weights
// C_j = sum_{k>=j} c_k (see launch_fd_step).
__device__ __forceinline__ float2 lap2(const float2 (&dz)[8], const float2 (&e)[8],
                                       const float2 (&cz)[4], const float2 (&cx)[4]) {
  float2 l = __fmul2_rn(cz[0], sub2(dz[4], dz[3]));
  l = __ffma2_rn(cz[1], sub2(dz[5], dz[2]), l);
  l = __ffma2_rn(cz[2], sub2(dz[6], dz[1]), l);
  l = __ffma2_rn(cz[3], sub2(dz[7], dz[0]), l);
  l = __ffma2_rn(cx[0], sub2(e[4], e[3]), l);
  l = __ffma2_rn(cx[1], sub2(e[5], e[2]), l);
  l = __ffma2_rn(cx[2], sub2(e[6], e[1]), l);
  l = __ffma2_rn(cx[3], sub2(e[7], e[0]), l);
  return l;
}

// A CTA holds one warp per receiver pair of the batch (threadIdx.y = pair), all on the same
// 64-column x TZ-row tile, so the coefficient rows are read from L2 once and served to the other
// pairs from L1.
constexpr int FD_MAXPAIRS = 16;

template <int TZ>
__global__ void __launch_bounds__(32 * FD_MAXPAIRS, EGH_FD_MINB)
    k_fd_step(const float2* __restrict__ ucur, const float2* __restrict__ uprev,
              float2* __restrict__ unext, const float2* __restrict__ coef, int NZ, int NX, int PX,
              int org, long long pstride, Stencil C, SnapOut so) {
  extern __shared__ __align__(16) float4 ring_all[];  // [pairs][FD_RING][36]
  float4 (*ring)[36] = reinterpret_cast<float4 (*)[36]>(ring_all + threadIdx.y * FD_RING * 36);
  const int lane = threadIdx.x;
  const int pair = threadIdx.y;
  const int x0 = blockIdx.x * 64;
  const int x = x0 + 2 * lane;  // this lane's first point
  const int z0 = blockIdx.y * TZ;
  const int nrows = min(TZ, NZ - z0);
  const int PX2 = PX >> 1;
  const int xh = x >> 1;
  const long long boff = (long long)pair * pstride + org;  // even: float4-aligned
  const float4* __restrict__ uc = reinterpret_cast<const float4*>(ucur + boff);
  const float4* __restrict__ up = reinterpret_cast<const float4*>(uprev + boff) + xh;
  float4* __restrict__ un = reinterpret_cast<float4*>(unext + boff) + xh;
  const float4* __restrict__ cf = reinterpret_cast<const float4*>(coef + org) + xh;
  const bool halo = lane < 2 || lane >= 30;
  const int hcol = lane < 2 ? (x0 >> 1) - 2 + lane : (x0 >> 1) + 32 + (lane - 30);
  const int hslot = lane < 2 ? lane : 34 + (lane - 30);
  const unsigned ring0 = (unsigned)__cvta_generic_to_shared(&ring[0][0]);
  const bool ok0 = x < NX, ok1 = x + 1 < NX;
  // ring row k holds u^n row z0 - 4 + k; rows z0 - 4 .. z0 + nrows + 3 exist (guard rows included)
  const int nload = nrows + 8;
  auto load_row = [&](int k) {
    if (k < nload) {
      const int z = z0 - 4 + k;
      const int r = z * PX2;
      const unsigned dst = ring0 + (unsigned)((k % FD_RING) * 36) * 16u;
      cp_async16(dst + (unsigned)(lane + 2) * 16u, uc + r + xh);
      // halo columns are read only for rows that are computed (0 <= z < NZ): there they stay
      // inside the level (previous row's padding, next row's first columns); a guard row's halo
      // would reach past the level
      if (halo && z >= 0 && z < NZ) cp_async16(dst + (unsigned)hslot * 16u, uc + r + hcol);
    }
    cp_async_commit();  // empty groups keep the group count uniform
  };
#pragma unroll
  for (int k = 0; k < FD_RING; ++k) load_row(k);
  float4 pu[FD_P], pc[FD_P];
#pragma unroll
  for (int i = 0; i < FD_P; ++i) {
    if (i < nrows) {
      pu[i] = __ldcg(up + (z0 + i) * PX2);
      pc[i] = __ldg(cf + (z0 + i) * PX2);
    }
  }
  cp_async_wait<FD_RING - 8>();  // rows 0 .. 7 have landed
  __syncwarp();
  // z first differences of both receivers at point p (0: x, 1: x + 1) of the lane:
  // dz[p][m] = D at row z - 3 + m for the current row z; ul = u^n at row z + 3
  float2 cz2[4], cx2[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    cz2[j] = make_float2(C.cz[j], C.cz[j]);
    cx2[j] = make_float2(C.cx[j], C.cx[j]);
  }
  float2 dz[2][8], ul[2];
  {
    const float4 v = ring[0][lane + 2];
    ul[0] = make_float2(v.x, v.y);
    ul[1] = make_float2(v.z, v.w);
  }
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const float4 v = ring[k][lane + 2];
    const float2 nv[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      dz[p][k] = sub2(nv[p], ul[p]);
      ul[p] = nv[p];
    }
  }
  __syncwarp();  // ring rows 0 .. 2 are refilled next
#pragma unroll
  for (int k = FD_RING; k < FD_D + 8; ++k) load_row(k);
  __nv_bfloat16* sbase = so.lvl ? so.lvl + (long long)(2 * pair) * so.rec + x : nullptr;
#pragma unroll
  for (int i = 0; i < TZ; ++i) {
    if (i >= nrows) break;
    // row i + 8 (z + 4) was committed FD_D groups ago
    load_row(FD_D + 8 + i);
    cp_async_wait<FD_D>();
    __syncwarp();
    const float4 uo = pu[i % FD_P], cc = pc[i % FD_P];
    if (i + FD_P < nrows) {
      pu[i % FD_P] = __ldcg(up + (z0 + i + FD_P) * PX2);
      pc[i % FD_P] = __ldg(cf + (z0 + i + FD_P) * PX2);
    }
    {
      const float4 v = ring[(i + 8) % FD_RING][lane + 2];  // u^n at row z + 4
      const float2 nv[2] = {make_float2(v.x, v.y), make_float2(v.z, v.w)};
#pragma unroll
      for (int p = 0; p < 2; ++p) {
#pragma unroll
        for (int m = 0; m < 7; ++m) dz[p][m] = dz[p][m + 1];
        dz[p][7] = sub2(nv[p], ul[p]);
        ul[p] = nv[p];
      }
    }
    const float4* xr = ring[(i + 4) % FD_RING];  // u^n at row z, points x0 - 4 .. x0 + 67
    const float4 A0 = xr[lane], A1 = xr[lane + 1], A2 = xr[lane + 2], A3 = xr[lane + 3],
                 A4 = xr[lane + 4];
    __syncwarp();  // every lane has read ring row i + 4 before it is refilled
    // both receivers at points x - 4 .. x + 5
    const float2 w[10] = {make_float2(A0.x, A0.y), make_float2(A0.z, A0.w), make_float2(A1.x, A1.y),
                          make_float2(A1.z, A1.w), make_float2(A2.x, A2.y), make_float2(A2.z, A2.w),
                          make_float2(A3.x, A3.y), make_float2(A3.z, A3.w), make_float2(A4.x, A4.y),
                          make_float2(A4.z, A4.w)};
    float2 e[9];
#pragma unroll
    for (int m = 0; m < 9; ++m) e[m] = sub2(w[m + 1], w[m]);
    const int z = z0 + i;
    float2 v0, v1;
    {
      const float2 e0[8] = {e[0], e[1], e[2], e[3], e[4], e[5], e[6], e[7]};
      const float2 e1[8] = {e[1], e[2], e[3], e[4], e[5], e[6], e[7], e[8]};
      const float2 l0 = lap2(dz[0], e0, cz2, cx2), l1 = lap2(dz[1], e1, cz2, cx2);
      // u^{n+1} = c3 L u + c1 (u - u^{n-1}) + u^{n-1}
      const float2 o0 = make_float2(uo.x, uo.y), o1 = make_float2(uo.z, uo.w);
      v0 = __ffma2_rn(make_float2(cc.y, cc.y), l0,
                      __ffma2_rn(make_float2(cc.x, cc.x), sub2(w[4], o0), o0));
      v1 = __ffma2_rn(make_float2(cc.w, cc.w), l1,
                      __ffma2_rn(make_float2(cc.z, cc.z), sub2(w[5], o1), o1));
      if (!ok1) v1 = make_float2(0.f, 0.f);
    }
    if (ok0) {
      un[z * PX2] = make_float4(v0.x, v0.y, v1.x, v1.y);
      if (sbase) {
        unsigned ha, la, hb, lb;
        split_bf16(v0.x, v1.x, ha, la);
        split_bf16(v0.y, v1.y, hb, lb);
        __nv_bfloat16* sp = sbase + z * PX;
        __stcs(reinterpret_cast<unsigned*>(sp), ha);
        __stcs(reinterpret_cast<unsigned*>(sp + so.plane), la);
        __stcs(reinterpret_cast<unsigned*>(sp + so.rec), hb);
        __stcs(reinterpret_cast<unsigned*>(sp + so.rec + so.plane), lb);
      }
    }
  }
  asm volatile("cp.async.wait_all;" ::: "memory");
}

#ifndef EGH_FD_TZDEF
#define EGH_FD_TZDEF 20
#endif

int fd_rows_per_warp_default() { return EGH_FD_TZDEF; }

int fd_block_smem(int npairs) { return (int)(sizeof(float4) * FD_RING * 36 * npairs); }

long long fd_sm_smem(int npairs, int tz) {
  int dev = 0, occ = 0, reserved = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev) != cudaSuccess)
    return 0;
  const void* k = nullptr;
  switch (tz) {
    case 12: k = (const void*)k_fd_step<12>; break;
    case 16: k = (const void*)k_fd_step<16>; break;
    case 18: k = (const void*)k_fd_step<18>; break;
    case 20: k = (const void*)k_fd_step<20>; break;
    case 24: k = (const void*)k_fd_step<24>; break;
    case 32: k = (const void*)k_fd_step<32>; break;
    default: k = (const void*)k_fd_step<EGH_FD_TZDEF>; break;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, 32 * npairs, fd_block_smem(npairs)) !=
      cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return (long long)occ * (fd_block_smem(npairs) + reserved);
}

// Rows per warp that fill one wave: the smallest choice whose tiles (PX/64 x ceil(NZ / TZ) CTAs)
// all fit the GPU's resident CTA slots at once, so that no SM carries more rows than another;
// the library default if none does.
int fd_rows_one_wave(const Layout& L, int npairs) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return EGH_FD_TZDEF;
  const size_t smem = fd_block_smem(npairs);
  const int threads = 32 * npairs;
  auto fits = [&](auto kern, int tz) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, threads, smem) != cudaSuccess)
      return false;
    return (long long)(L.PX / 64) * ((L.NZ + tz - 1) / tz) <= (long long)occ * sms;
  };
  if (fits(k_fd_step<12>, 12)) return 12;
  if (fits(k_fd_step<16>, 16)) return 16;
  if (fits(k_fd_step<18>, 18)) return 18;
  if (fits(k_fd_step<20>, 20)) return 20;
  if (fits(k_fd_step<24>, 24)) return 24;
  if (fits(k_fd_step<32>, 32)) return 32;
  return EGH_FD_TZDEF;
}

// Raises the dynamic shared-memory limit of every FD and transform kernel instance once per
// process (outside any stream capture).
cudaError_t fd_prepare(int nf) {
  const int fd_smem = (int)(sizeof(float4) * FD_RING * 36 * FD_MAXPAIRS);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_fd_step<12>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  if ((e = cudaFuncSetAttribute(k_fd_step<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  if ((e = cudaFuncSetAttribute(k_fd_step<18>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  if ((e = cudaFuncSetAttribute(k_fd_step<20>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  if ((e = cudaFuncSetAttribute(k_fd_step<24>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  if ((e = cudaFuncSetAttribute(k_fd_step<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, fd_smem))) return e;
  // the FD steps and the transform beside them share each SM's shared memory: ask for all of it
  for (const void* f : {(const void*)k_fd_step<12>, (const void*)k_fd_step<16>, (const void*)k_fd_step<18>,
                        (const void*)k_fd_step<20>, (const void*)k_fd_step<24>, (const void*)k_fd_step<32>})
    if ((e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                  (int)cudaSharedmemCarveoutMaxShared)))
      return e;
  (void)nf;
  return cudaSuccess;
}

cudaError_t launch_fd_step(const float2* ucur, const float2* uprev, float2* unext,
                           const float2* coef, const Layout& L, const Stencil& S, int npairs,
                           const SnapOut& so, cudaStream_t st, int tz) {
  if (L.PX % 64 != 0) return cudaErrorInvalidValue;
  if (tz <= 0) tz = EGH_FD_TZDEF;
  // cumulative weights C_j = sum_{k>=j} c_k of the first-difference form
  Stencil C;
  float az = 0.f, ax = 0.f;
  for (int k = 3; k >= 0; --k) {
    az += S.cz[k];
    ax += S.cx[k];
    C.cz[k] = az;
    C.cx[k] = ax;
  }
  if (npairs < 1 || npairs > FD_MAXPAIRS) return cudaErrorInvalidValue;
  count_launches(1);
  const dim3 blk(32, npairs);
  const size_t smem = fd_block_smem(npairs);
  const int org = (int)L.org;
  switch (tz) {
#define EGH_FD_CASE(T)                                                                          \
  case T:                                                                                       \
    k_fd_step<T><<<dim3(L.PX / 64, (L.NZ + T - 1) / T), blk, smem, st>>>(                        \
        ucur, uprev, unext, coef, L.NZ, L.NX, L.PX, org, L.F, C, so);                           \
    break;
    EGH_FD_CASE(12)
    EGH_FD_CASE(16)
    EGH_FD_CASE(18)
    EGH_FD_CASE(20)
    EGH_FD_CASE(24)
    EGH_FD_CASE(32)
#undef EGH_FD_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Point sources on paired levels: receiver b is lane b % 2 of pair b / 2.
//   u[b][pts[b]] += c3[pts[b]] * amp * scale   (source term dt^2 v^2 f^n / (1 + a), f^n = amp/(dx dz))
// With `so.lvl` set, the new value's hi/lo split is also written to the snapshot slot (used for
// level 1 of a Green-function batch, the impulse, whose slot holds zeros).
// ---------------------------------------------------------------------------------------------
__global__ void k_inject(float2* __restrict__ u, long long pstride, const int* __restrict__ pts,
                         const float2* __restrict__ coef, int nb, float amp, float scale,
                         long long org, SnapOut so) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int p = pts[b];
  float* v = reinterpret_cast<float*>(u + (long long)(b >> 1) * pstride + p) + (b & 1);
  const float nv = *v + coef[p].y * amp * scale;
  *v = nv;
  if (so.lvl) {
    const __nv_bfloat16 h = __float2bfloat16_rn(nv);
    const __nv_bfloat16 l = __float2bfloat16_rn(nv - __bfloat162float(h));
    __nv_bfloat16* s = so.lvl + (long long)b * so.rec + (p - org);
    s[0] = h;
    s[so.plane] = l;
  }
}

cudaError_t launch_inject(float2* u, long long pstride, const int* pts, const float2* coef, int nb,
                          float amp, float scale, long long org, const SnapOut& so,
                          cudaStream_t st) {
  count_launches(1);
  k_inject<<<(nb + 127) / 128, 128, 0, st>>>(u, pstride, pts, coef, nb, amp, scale, org, so);
  return cudaGetLastError();
}

// traces[b][r][t] = receiver b's level at rec_pts[r]  (offsets inside a level)
__global__ void k_record(const float2* __restrict__ u, long long pstride,
                         const int* __restrict__ rec_pts, int nrec, int nb,
                         float* __restrict__ traces, int nt, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrec * nb) return;
  const int b = i / nrec, r = i % nrec;
  const float2 v = u[(long long)(b >> 1) * pstride + rec_pts[r]];
  traces[((long long)b * nrec + r) * nt + t] = (b & 1) ? v.y : v.x;
}

cudaError_t launch_record(const float2* u, long long pstride, const int* rec_pts, int nrec, int nb,
                          float* traces, int nt, int t, cudaStream_t st) {
  const int n = nrec * nb;
  count_launches(1);
  k_record<<<(n + 255) / 256, 256, 0, st>>>(u, pstride, rec_pts, nrec, nb, traces, nt, t);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// On-the-fly transform of one chunk of levels n0 .. n0+kcount-1 of a batch, on the tensor cores:
//     gh[rec][c][p] (+)= sum_j u^{n0+j}[rec][p] W[c][n0+j],   W[2k][n] = cos(2 pi f_k n dt),
//                                                             W[2k+1][n] = -sin(2 pi f_k n dt),
// in bf16x3: u = u_hi + u_lo (split by the FD step), W = W_hi + W_lo (split on the host), and
// u_hi W_hi + u_hi W_lo + u_lo W_hi accumulated in FP32 in TMEM (the dropped u_lo W_lo and the
// splits themselves are ~2^-17 relative).  The chunk that ends the record also writes the final
// transforms' bf16 hi/lo split (the Gram's operands).  One tile is D = A B^T for 128 points of
// one receiver: M = 128, N = 2 nf rounded up to 32, K = the chunk's levels in stages of 32.
// A (snapshots) is MN-major: a 4-D TMA box {64 points, 1 receiver, 32 levels, 2 planes} lands as
// [plane][level][64 points] 128-byte rows with the 128-byte swizzle (two boxes per stage).
// B (twiddles) is K-major in host-swizzled tiles of 64 levels (one 128-byte row per component),
// one 1-D bulk copy per tile.
//
// The kernel is persistent and small so that it runs BESIDE the FD steps of the next chunk: one
// CTA per SM (a fixed grid of at most one CTA per SM walks the tiles), 128 threads at 32
// registers and 66.5 KB of shared memory, which fit next to the two FD CTAs an SM holds (2 x 256
// threads x 120 registers, 2 x 55 KB).  Launched as a grid of thousands of short CTAs, the
// transform's CTAs took whole SMs between FD launches and the FD steps waited for them, so that
// the two ran one after the other; side by side they share the SMs, and the FD steps, which are
// bound by issue and latency, lose less than the transform's run time.
// One thread issues the copies and the MMAs over a ring of nring stages (3 beside the FD steps,
// where the padded shared memory has room; 2 alone): the copies of stage s + nring are issued
// once the MMAs of stage s are done, which with two twiddle buffers (one per 64 levels) keeps a
// twiddle buffer from being refilled while MMAs still read it for nring <= 3.  After a tile's
// last stage
// every thread reads its point's row of TMEM in groups of 8 columns and adds it into gh (plain
// store for the chunk that starts at level 0).  Every mbarrier wait is bounded: on expiry the
// CTA records the error flag, waits (bounded) for its copies and MMAs in flight, frees its TMEM
// and leaves.
// ---------------------------------------------------------------------------------------------
constexpr int TD_M = 128;                // points per tile (MMA M)
constexpr int TD_S = 32;                 // levels per stage
constexpr int TD_STMAX = 3;              // stages in flight at most
constexpr unsigned TD_AB = 16384;        // one stage of A: 2 atoms x 2 planes x 32 x 128 B
constexpr int TD_NMAX = 128;             // largest N (TMEM columns: N rounded up to a power of two)

int dft_ncomp(int nf) { return (2 * nf + 31) / 32 * 32; }

// dynamic shared memory for a ring of nring stages
size_t dft_smem_ring(int nf, int nring) {
  return 1024 + (size_t)nring * TD_AB + 2 * 2 * (size_t)dft_ncomp(nf) * 128;
}
size_t dft_smem(int nf) { return dft_smem_ring(nf, 2); }

__device__ __forceinline__ void tmem_ld8(unsigned taddr, float (&v)[8]) {
  unsigned q[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(q[0]), "=r"(q[1]), "=r"(q[2]), "=r"(q[3]), "=r"(q[4]), "=r"(q[5]), "=r"(q[6]),
                 "=r"(q[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(q[i]);
}

__global__ void __launch_bounds__(128, 16)
    k_dft_tc(const __grid_constant__ CUtensorMap tmap, const unsigned char* __restrict__ twt,
             int N, int nf, int slot0, int kcount, int n0, long long G, float* __restrict__ gh,
             __nv_bfloat16* __restrict__ ghb, int last, int rec0, int nvalid, int nrec_all,
             int* __restrict__ err, int expire, int nring) {
  extern __shared__ __align__(1024) unsigned char dsm[];
  unsigned char* sm = dsm + ((1024 - (tc::smem_u32(dsm) & 1023)) & 1023);
  unsigned char* As = sm;                       // [nring][TD_AB]
  unsigned char* Bs = sm + nring * TD_AB;       // [2][plane][N][128 B]
  const unsigned tile = 2u * (unsigned)N * 128u;
  __shared__ __align__(8) unsigned long long bars[2 * TD_STMAX + 2];  // full[], empty[], done, never
  __shared__ unsigned tslot;
  __shared__ int fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  // N <= 64: A hi against the twiddles' hi and lo planes as one MMA of width 2N, then A lo
  // against hi; columns [0, N) hold hi.hi + lo.hi and [N, 2N) hi.lo.  Wider N: three MMAs of
  // width N (2N columns would not fit three CTAs' TMEM on one SM).
  const bool two = N <= 64;
  const unsigned ncols = N <= 32 ? 64u : N <= 64 ? 128u : 128u;
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  const unsigned bar0 = tc::smem_u32(&bars[0]);
  auto full = [&](int i) { return bar0 + 8u * i; };
  auto empty = [&](int i) { return bar0 + 8u * (TD_STMAX + i); };
  const unsigned done = bar0 + 8u * (2 * TD_STMAX);
  if (tid == 0) {
    for (int i = 0; i < 2 * TD_STMAX + 2; ++i) tc::mbar_init(bar0 + 8u * i, 1);
    fail = 0;
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  const int npb = (int)(G / TD_M);       // 128-point blocks
  const int ntile = npb * nvalid;        // tiles: block-major within a receiver
  const int nst = (kcount + TD_S - 1) / TD_S;
  const bool first = n0 == 0;
  // stage q of this CTA (counted over all its tiles) uses buffer q % nring in phase (q / nring) & 1
  int q0 = 0, it = 0;
  for (int t = blockIdx.x; t < ntile; t += gridDim.x, ++it, q0 += nst) {
    const int r = t / npb;
    const int p0 = (t - r * npb) * TD_M;
    if (tid == 0) {
      const unsigned idesc = tc::idesc_bf16(TD_M, N, 1, 0), idesc2 = tc::idesc_bf16(TD_M, 2 * N, 1, 0);
      // snapshots are read once: stream them through L2 as evict-first so that the FD's state
      // levels, which the concurrent FD steps re-read, stay resident
      const uint64_t pol = tc::l2_evict_first_policy();
      auto issue = [&](int s) {
        const int buf = (q0 + s) % nring;
        const int n = n0 + s * TD_S;
        const bool newtile = s == 0 || (n & 63) == 0;
        tc::mbar_expect_tx(full(buf), TD_AB + (newtile ? tile : 0u));
        for (int m = 0; m < 2; ++m)
          tc::tma_load_4d_hint(tc::smem_u32(As + buf * TD_AB + m * 8192), &tmap, p0 + 64 * m, r,
                               slot0 + s * TD_S, 0, full(buf), pol);
        if (newtile)
          tc::bulk_g2s(tc::smem_u32(Bs + ((n >> 6) & 1) * tile), twt + (size_t)(n >> 6) * tile, tile,
                       full(buf));
      };
      int issued = 0, landed = 0;
      bool ok = true;
      for (; issued < min(nst, nring); ++issued) issue(issued);
      // test hook: the first CTA's first wait runs out (the last barrier never completes a phase)
      if (expire && blockIdx.x == 0 && it == 0 &&
          !tc::mbar_wait_unsignalled(bar0 + 8u * (2 * TD_STMAX + 1)))
        ok = false;
      for (int s = 0; ok && s < nst; ++s) {
        const int q = q0 + s;
        const int buf = q % nring;
        if (!tc::mbar_wait(full(buf), (q / nring) & 1)) {
          ok = false;
          break;
        }
        landed = s + 1;
        tc::tc_fence_after();
        const int n = n0 + s * TD_S;
        const unsigned bh = tc::smem_u32(Bs + ((n >> 6) & 1) * tile) + (unsigned)(n & 63) * 2u;
        const unsigned bl = bh + (unsigned)N * 128u;
        const unsigned ab = tc::smem_u32(As + buf * TD_AB);
#pragma unroll
        for (int ks = 0; ks < 2; ++ks) {
          const uint64_t ahi = tc::sdesc_sw128_lbo_sbo(ab + ks * 2048, 8192, 1024);
          const uint64_t alo = tc::sdesc_sw128_lbo_sbo(ab + 4096 + ks * 2048, 8192, 1024);
          const uint64_t bhi = tc::sdesc_sw128(bh + ks * 32), blo = tc::sdesc_sw128(bl + ks * 32);
          if (two) {  // the lo plane is rows N .. 2N - 1 of the same K-major tile
            tc::mma_bf16(tmem, ahi, bhi, idesc2, s > 0 || ks > 0);
          } else {
            tc::mma_bf16(tmem, ahi, bhi, idesc, s > 0 || ks > 0);
            tc::mma_bf16(tmem, ahi, blo, idesc, true);
          }
          tc::mma_bf16(tmem, alo, bhi, idesc, true);
        }
        tc::mma_commit(empty(buf));
        if (issued < nst) {  // the next stage to issue reuses this stage's buffer
          if (!tc::mbar_wait(empty(buf), (q / nring) & 1)) {
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
        // let the copies in flight land (bounded) before the CTA leaves
        for (int s = landed; s < issued; ++s)
          tc::mbar_wait(full((q0 + s) % nring), ((q0 + s) / nring) & 1);
      }
      tc::mma_commit(done);  // arrives once every MMA issued so far has completed
    }
    __syncwarp();
    const bool okd = tc::mbar_wait(done, it & 1);
    if (__syncthreads_or(!okd || (tid == 0 && fail))) {
      if (tid == 0) atomicExch(err, 1);
      break;
    }
    tc::tc_fence_after();
    const long long p = p0 + tid;
    const long long row0 = (long long)(rec0 + r) * 2 * nf;  // first plane of this receiver
    float* g = gh + row0 * G + p;
    for (int c0 = 0; c0 < N; c0 += 8) {
      float v[8], o[8];
      tmem_ld8(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0, v);
      if (two) {  // the hi.lo columns, through o before o takes the old totals
        tmem_ld8(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(N + c0), o);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] += o[i];
      }
      // all loads of the group before any store: the 8 column planes are distinct
#pragma unroll
      for (int i = 0; i < 8; ++i)
        o[i] = (!first && c0 + i < 2 * nf) ? __ldcs(g + (long long)(c0 + i) * G) : 0.f;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = c0 + i;
        if (c < 2 * nf) {
          const float sum = o[i] + v[i];
          __stcs(g + (long long)c * G, sum);
          if (last) {
            // the Gram's operands: hi = bf16(g), lo = bf16(g - hi), blocked by 64 points as
            // [freq][G/64][hi|lo][receiver, re/im][64] (each 64-receiver box is contiguous)
            const __nv_bfloat16 h = __float2bfloat16_rn(sum);
            const __nv_bfloat16 l = __float2bfloat16_rn(sum - __bfloat162float(h));
            const long long rows = 2LL * nrec_all;
            __nv_bfloat16* qp = ghb + (((long long)(c >> 1) * (G >> 6) + (p >> 6)) * 2 * rows +
                                       2LL * (rec0 + r) + (c & 1)) * 64 + (p & 63);
            qp[0] = h;
            qp[rows * 64] = l;
          }
        }
      }
    }
    // every thread has read TMEM before the next tile's first MMA overwrites it
    tc::tc_fence_before();
    __syncthreads();
    tc::tc_fence_after();
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

cudaError_t launch_dft_tc(const CUtensorMap& tmap, const unsigned char* twt, int nf, int slot0,
                          int kcount, int n0, const Layout& L, float* gh, __nv_bfloat16* ghb,
                          int last, int rec0, int nvalid, int nrec_all, int* err, int expire,
                          int per_sm, long long beside_smem, cudaStream_t st) {
  const int N = dft_ncomp(nf);
  if (L.G % TD_M != 0 || N > TD_NMAX || kcount < 1 || slot0 % TD_S != 0 || n0 % TD_S != 0 ||
      nvalid < 1 || per_sm < 0 || per_sm > 3 || beside_smem < 0)
    return cudaErrorInvalidValue;
  cudaError_t e;
  int dev = 0, sms = 0, sm_smem = 0, reserved = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
      (e = cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev)) !=
          cudaSuccess ||
      (e = cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev)) !=
          cudaSuccess)
    return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, k_dft_tc)) != cudaSuccess) return e;
  int nring = 2;
  size_t smem = dft_smem_ring(nf, 2);
  if (beside_smem > 0) {
    // Beside the FD CTAs an SM holds (beside_smem bytes of shared memory in all, reserved parts
    // included): the largest size that still fits there, if that size also keeps a second
    // transform CTA off the SM.  A CTA per SM is then all an SM can take, wherever the launch
    // finds free room (at a chunk boundary, SMs whose FD CTAs have left would otherwise take two
    // or three and hold back the next FD step).  The padded size holds a third stage where it
    // has room: one CTA per SM keeps three copies in flight.
    const long long cta = (long long)fa.sharedSizeBytes + reserved;
    const long long fit = (long long)sm_smem - beside_smem - cta;
    if (fit >= (long long)smem && 2 * (fit + cta) > sm_smem) {
      smem = (size_t)fit;
      if ((long long)dft_smem_ring(nf, 3) <= fit) nring = 3;
    }
  }
  if ((e = cudaFuncSetAttribute(k_dft_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ||
      (e = cudaFuncSetAttribute(k_dft_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                                (int)cudaSharedmemCarveoutMaxShared)))
    return e;
  // a persistent grid (per_sm > 0) must be resident at once: at most the SM's occupancy; per_sm
  // = 0 launches one CTA per tile
  int occ = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_dft_tc, 128, smem)) != cudaSuccess)
    return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long ntile = (L.G / TD_M) * nvalid;
  const int grid = (int)(per_sm == 0 ? ntile
                                     : std::min<long long>((long long)sms * std::min(per_sm, occ), ntile));
  count_launches(1);
  k_dft_tc<<<grid, 128, smem, st>>>(tmap, twt, N, nf, slot0, kcount, n0, L.G, gh, ghb, last, rec0,
                                    nvalid, nrec_all, err, expire, nring);
  return cudaGetLastError();
}

// Twiddle tiles for k_dft_tc: for every 64 levels, a hi tile and a lo tile of [N][64] bf16 in the
// 128-byte-swizzled K-major layout (row c, level j at byte (c/8)*1024 + (c%8)*128 +
// (((2j/16) ^ (c%8)) * 16) + 2j%16); row 2k = cos(2 pi f_k n dt), row 2k+1 = -sin(2 pi f_k n dt)
// with the phase reduced as 2 pi frac(f_k n dt) in double precision; hi = bf16(w),
// lo = bf16(w - hi); rows >= 2 nf and levels >= nt are zero.  With `scale`, row pair k holds
// Re and Im of scale[k] exp(-i 2 pi f_k n dt) instead (the band-limited, decimated form folds its
// decimation factor and spectral division into the twiddles).
std::vector<unsigned char> dft_twiddle_tiles(const std::vector<double>& f, double dt, int nt,
                                             const std::vector<std::complex<double>>* scale) {
  const int nf = (int)f.size(), N = dft_ncomp(nf);
  const int ntile = (nt + 63) / 64;
  const size_t tile = 2ull * N * 128;
  std::vector<unsigned char> out((size_t)ntile * tile, 0);
  for (int n = 0; n < nt; ++n) {
    unsigned char* hi = out.data() + (size_t)(n / 64) * tile;
    unsigned char* lo = hi + (size_t)N * 128;
    const int j = n % 64;
    for (int k = 0; k < nf; ++k) {
      double ph = f[k] * (double)n * dt;
      ph -= std::floor(ph);
      const double a = 2.0 * M_PI * ph;
      std::complex<double> w(std::cos(a), -std::sin(a));
      if (scale) w *= (*scale)[k];
      const double v[2] = {w.real(), w.imag()};
      for (int q = 0; q < 2; ++q) {
        const int c = 2 * k + q;
        const size_t off = (size_t)(c >> 3) * 1024 + (c & 7) * 128 +
                           ((((2 * j) >> 4) ^ (c & 7)) << 4) + ((2 * j) & 15);
        const __nv_bfloat16 h = __float2bfloat16_rn((float)v[q]);
        const __nv_bfloat16 l = __float2bfloat16_rn((float)(v[q] - (double)__bfloat162float(h)));
        std::memcpy(hi + off, &h, 2);
        std::memcpy(lo + off, &l, 2);
      }
    }
  }
  return out;
}

// Tensor map of the snapshot ring [2 planes][nslot][Bp receivers][G] bf16 for k_dft_tc's boxes
// {64 points, 1 receiver, 32 levels, 2 planes} with the 128-byte swizzle.
cudaError_t make_snap_tmap(CUtensorMap* tm, void* base, long long G, int Bp, int nslot) {
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
  const cuuint64_t dims[4] = {(cuuint64_t)G, (cuuint64_t)Bp, (cuuint64_t)nslot, 2};
  const cuuint64_t str[3] = {(cuuint64_t)G * 2, (cuuint64_t)G * 2 * Bp,
                             (cuuint64_t)G * 2 * Bp * nslot};
  const cuuint32_t box[4] = {64, 1, (cuuint32_t)TD_S, 2};
  const cuuint32_t es[4] = {1, 1, 1, 1};
  const CUresult r = enc(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, str, box, es,
                         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                         CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

}  // namespace egh
