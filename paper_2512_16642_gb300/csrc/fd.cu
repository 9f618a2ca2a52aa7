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
#include <cfloat>
#include <cmath>

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
// One leapfrog step for a batch of receiver pairs.  Each warp owns 32 columns of one pair and
// marches down FD_TZ rows (fully unrolled, so the nine z-neighbours of its column rotate through
// registers without moves); the x-neighbours come from a 40-entry row staged in shared memory
// (32 + 4 halo on each side).  Rows are processed in groups of FD_U whose loads are all issued
// before the group is computed.  Reads of guard rows and padding columns return the zero
// boundary, so there is no bounds test on loads; rows past the warp's range are not loaded.
// ---------------------------------------------------------------------------------------------
constexpr int FD_WARPS = 4;
constexpr int FD_TZ = 16;
constexpr int FD_U = 4;

__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);  // a - b, one rounding
}

__global__ void __launch_bounds__(32 * FD_WARPS)
    k_fd_step(const float2* __restrict__ ucur, const float2* __restrict__ uprev,
              float2* __restrict__ unext, const float2* __restrict__ coef, int NZ, int NX, int PX,
              int org, long long pstride, Stencil S) {
  __shared__ float2 srow[FD_WARPS][40];
  const int lane = threadIdx.x;
  const int w = threadIdx.y;
  const int x0 = blockIdx.x * 32;
  const int x = x0 + lane;
  const int z0 = (blockIdx.y * FD_WARPS + w) * FD_TZ;
  if (z0 >= NZ) return;  // whole warp leaves; only warp-level synchronisation below
  const long long boff = (long long)blockIdx.z * pstride + org;
  const float2* __restrict__ uc = ucur + boff;
  const float2* __restrict__ up = uprev + boff;
  float2* __restrict__ un = unext + boff;
  const float2* __restrict__ cf = coef + org;
  const bool halo = lane < 4 || lane >= 28;
  const int hcol = lane < 4 ? x0 - 4 + lane : x0 + 4 + lane;
  const int hslot = lane < 4 ? lane : lane + 8;
  float2* row = srow[w];
  const float2 cz0 = make_float2(S.cz[0], S.cz[0]), cz1 = make_float2(S.cz[1], S.cz[1]);
  const float2 cz2 = make_float2(S.cz[2], S.cz[2]), cz3 = make_float2(S.cz[3], S.cz[3]);
  const float2 cx0 = make_float2(S.cx[0], S.cx[0]), cx1 = make_float2(S.cx[1], S.cx[1]);
  const float2 cx2 = make_float2(S.cx[2], S.cx[2]), cx3 = make_float2(S.cx[3], S.cx[3]);

  float2 q[9];
  const int o0 = (z0 - 4) * PX + x;
#pragma unroll
  for (int i = 0; i < 8; ++i) q[i + 1] = uc[o0 + i * PX];
  const int nrows = min(FD_TZ, NZ - z0);
#pragma unroll
  for (int g = 0; g < FD_TZ; g += FD_U) {
    float2 qn[FD_U], hv[FD_U], uo[FD_U], cc[FD_U];
#pragma unroll
    for (int i = 0; i < FD_U; ++i) {
      if (g + i < nrows) {
        const int r = (z0 + g + i) * PX;
        cc[i] = cf[r + x];
        qn[i] = uc[r + 4 * PX + x];
        uo[i] = up[r + x];
        hv[i] = halo ? uc[r + hcol] : make_float2(0.f, 0.f);
      }
    }
#pragma unroll
    for (int i = 0; i < FD_U; ++i) {
      if (g + i >= nrows) return;
#pragma unroll
      for (int j = 0; j < 8; ++j) q[j] = q[j + 1];
      q[8] = qn[i];
      row[lane + 4] = q[4];
      if (halo) row[hslot] = hv[i];
      __syncwarp();
      if (x < NX) {
        // Laplacian as sum_k c_k [(u_{+k} - u) + (u_{-k} - u)] (c_0 = -2 sum_k c_k): neighbour
        // differences of a well-sampled field are exact in float32, so the large cancelling
        // terms of c_0 u + sum_k c_k (u_{+k} + u_{-k}) never form.
        const float2 u0 = q[4];
        float2 lap = __fmul2_rn(cz0, __fadd2_rn(sub2(q[3], u0), sub2(q[5], u0)));
        lap = __ffma2_rn(cz1, __fadd2_rn(sub2(q[2], u0), sub2(q[6], u0)), lap);
        lap = __ffma2_rn(cz2, __fadd2_rn(sub2(q[1], u0), sub2(q[7], u0)), lap);
        lap = __ffma2_rn(cz3, __fadd2_rn(sub2(q[0], u0), sub2(q[8], u0)), lap);
        lap = __ffma2_rn(cx0, __fadd2_rn(sub2(row[lane + 3], u0), sub2(row[lane + 5], u0)), lap);
        lap = __ffma2_rn(cx1, __fadd2_rn(sub2(row[lane + 2], u0), sub2(row[lane + 6], u0)), lap);
        lap = __ffma2_rn(cx2, __fadd2_rn(sub2(row[lane + 1], u0), sub2(row[lane + 7], u0)), lap);
        lap = __ffma2_rn(cx3, __fadd2_rn(sub2(row[lane + 0], u0), sub2(row[lane + 8], u0)), lap);
        const float2 c1 = make_float2(cc[i].x, cc[i].x), c3 = make_float2(cc[i].y, cc[i].y);
        un[(z0 + g + i) * PX + x] = __ffma2_rn(c3, lap, __ffma2_rn(c1, sub2(u0, uo[i]), uo[i]));
      }
      __syncwarp();
    }
  }
}

cudaError_t launch_fd_step(const float2* ucur, const float2* uprev, float2* unext,
                           const float2* coef, const Layout& L, const Stencil& S, int npairs,
                           cudaStream_t st) {
  dim3 block(32, FD_WARPS);
  const int rows = (L.NZ + FD_WARPS * FD_TZ - 1) / (FD_WARPS * FD_TZ);
  dim3 grid(L.PX / 32, rows, npairs);
  count_launches(1);
  k_fd_step<<<grid, block, 0, st>>>(ucur, uprev, unext, coef, L.NZ, L.NX, L.PX, (int)L.org, L.F,
                                    S);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Point sources on paired levels: receiver b is lane b % 2 of pair b / 2.
//   u[b][pts[b]] += c3[pts[b]] * amp * scale   (source term dt^2 v^2 f^n / (1 + a), f^n = amp/(dx dz))
// ---------------------------------------------------------------------------------------------
__global__ void k_inject(float2* __restrict__ u, long long pstride, const int* __restrict__ pts,
                         const float2* __restrict__ coef, int nb, float amp, float scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int p = pts[b];
  float* v = reinterpret_cast<float*>(u + (long long)(b >> 1) * pstride + p) + (b & 1);
  *v += coef[p].y * amp * scale;
}

cudaError_t launch_inject(float2* u, long long pstride, const int* pts, const float2* coef, int nb,
                          float amp, float scale, cudaStream_t st) {
  count_launches(1);
  k_inject<<<(nb + 127) / 128, 128, 0, st>>>(u, pstride, pts, coef, nb, amp, scale);
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
// On-the-fly transform of one chunk of kcount consecutive levels n0 .. n0+kcount-1 of a batch
// (ring slots slot0 .. slot0+kcount-1), on the tensor cores:
//     gh[rec][k][re/im][p] += sum_j tw[n0+j][k] * u^{n0+j}[rec][p]
// is the product D[p][c] = sum_j U[p][j] W[c][j] with c = 2k (cos row) / 2k+1 (-sin row),
// M = 128 points per block, N = 2 nf padded to 16, K = levels.  Per stage of 32 levels one
// thread brings the 32 level rows of the block's 128 points of a receiver pair (1-D bulk TMA
// copies) and the stage's pre-swizzled twiddle tiles into shared memory on an mbarrier
// (double-buffered); the threads transpose the levels into K-major 128-byte-swizzled tiles
// (point = row), splitting each value into tf32 hi + lo; one thread issues, per receiver,
// hi*hi + hi*lo + lo*hi (3xTF32) MMAs accumulating in TMEM (two N-column accumulators, one per
// receiver).  After the last stage the accumulators are read with tcgen05.ld and added into gh,
// which is therefore read and written once per chunk.  Every mbarrier wait is bounded; on expiry
// the block records the error flag, waits (bounded) for its copies and MMAs in flight, frees
// its TMEM and leaves.
// ---------------------------------------------------------------------------------------------
constexpr int T_P = 128;   // points per block (MMA M)
constexpr int T_SUB = 32;  // levels per stage (MMA K per stage)

int dft_ncomp(int nf) { return (2 * nf + 15) / 16 * 16; }

size_t dft_chunk_smem(int nf) {
  const int N = dft_ncomp(nf);
  return 1024 + sizeof(float2) * 2 * T_SUB * T_P + sizeof(float) * 4 * T_P * T_SUB +
         sizeof(float) * 2 * 2 * (size_t)N * T_SUB;
}

__global__ void __launch_bounds__(T_P)
    k_dft_chunk(const float2* __restrict__ ring, long long slot_stride, long long pstride,
                long long org, int slot0, int kcount, const float* __restrict__ twt, int stage0,
                int N, int nf, long long G, float* __restrict__ gh, int rec0, int nvalid,
                int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char dsm_raw[];
  unsigned char* sm = dsm_raw + ((1024 - (tc::smem_u32(dsm_raw) & 1023)) & 1023);
  float2* raw = reinterpret_cast<float2*>(sm);                      // [2][T_SUB][T_P]
  unsigned char* At = sm + sizeof(float2) * 2 * T_SUB * T_P;        // a_hi, a_lo, b_hi, b_lo
  unsigned char* Bt = At + sizeof(float) * 4 * T_P * T_SUB;         // [2][hi, lo][N][T_SUB]
  constexpr unsigned kAT = sizeof(float) * T_P * T_SUB;             // one A tile: 16 KB
  const unsigned kBT = sizeof(float) * N * T_SUB;                   // one twiddle tile
  __shared__ __align__(8) unsigned long long bars[3];               // stage[0], stage[1], mma
  __shared__ unsigned tslot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const unsigned ncols = 2 * N <= 32 ? 32u : 2 * N <= 64 ? 64u : 2 * N <= 128 ? 128u : 256u;
  if (warp == 0) tc::tmem_alloc(&tslot, ncols);
  const unsigned bst0 = tc::smem_u32(&bars[0]), bst1 = tc::smem_u32(&bars[1]);
  const unsigned bmma = tc::smem_u32(&bars[2]);
  if (tid == 0) {
    tc::mbar_init(bst0, 1);
    tc::mbar_init(bst1, 1);
    tc::mbar_init(bmma, 1);
    tc::mbar_init_fence();
  }
  tc::tc_fence_before();
  __syncthreads();
  tc::tc_fence_after();
  const unsigned tmem = tslot;
  const int pair = blockIdx.y;
  const long long p0 = (long long)blockIdx.x * T_P;
  const float2* src = ring + (long long)pair * pstride + org + p0;
  const int nst = (kcount + T_SUB - 1) / T_SUB;
  auto issue = [&](int s) {
    const int buf = s & 1, j0 = s * T_SUB, jn = min(T_SUB, kcount - j0);
    const unsigned bar = buf ? bst1 : bst0;
    tc::mbar_expect_tx(bar, (unsigned)(jn * T_P * sizeof(float2)) + 2 * kBT);
    for (int j = 0; j < jn; ++j)
      tc::bulk_g2s(tc::smem_u32(raw + (buf * T_SUB + j) * T_P),
                   src + (long long)(slot0 + j0 + j) * slot_stride, T_P * sizeof(float2), bar);
    tc::bulk_g2s(tc::smem_u32(Bt + buf * 2 * kBT), twt + (long long)(stage0 + s) * 2 * N * T_SUB,
                 2 * kBT, bar);
  };
  if (tid == 0) {
    issue(0);
    if (nst > 1) issue(1);
  }
  const unsigned idesc = tc::idesc_tf32(T_P, N);
  int s_fail = -1;
  for (int s = 0; s < nst; ++s) {
    const int buf = s & 1;
    bool ok = tc::mbar_wait(buf ? bst1 : bst0, (s >> 1) & 1);
    if (s > 0) ok = ok && tc::mbar_wait(bmma, (s - 1) & 1);  // the A tiles are free again
    if (__syncthreads_or(!ok)) {
      s_fail = s;
      break;
    }
    tc::tc_fence_after();
    const int jn = min(T_SUB, kcount - s * T_SUB);
    const float2* rb = raw + buf * T_SUB * T_P + tid;
#pragma unroll
    for (int jc = 0; jc < T_SUB / 4; ++jc) {
      float ax[4], bx[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = 4 * jc + e;
        const float2 v = j < jn ? rb[j * T_P] : make_float2(0.f, 0.f);
        ax[e] = v.x;
        bx[e] = v.y;
      }
      float4 ah, al, bh, bl;
      ah.x = tc::tf32_hi(ax[0]); ah.y = tc::tf32_hi(ax[1]); ah.z = tc::tf32_hi(ax[2]); ah.w = tc::tf32_hi(ax[3]);
      bh.x = tc::tf32_hi(bx[0]); bh.y = tc::tf32_hi(bx[1]); bh.z = tc::tf32_hi(bx[2]); bh.w = tc::tf32_hi(bx[3]);
      al = make_float4(ax[0] - ah.x, ax[1] - ah.y, ax[2] - ah.z, ax[3] - ah.w);
      bl = make_float4(bx[0] - bh.x, bx[1] - bh.y, bx[2] - bh.z, bx[3] - bh.w);
      const unsigned off = tc::sw128_offset(tid, 4 * jc);
      *reinterpret_cast<float4*>(At + 0 * kAT + off) = ah;
      *reinterpret_cast<float4*>(At + 1 * kAT + off) = al;
      *reinterpret_cast<float4*>(At + 2 * kAT + off) = bh;
      *reinterpret_cast<float4*>(At + 3 * kAT + off) = bl;
    }
    tc::fence_proxy_async();
    tc::tc_fence_before();
    __syncthreads();
    if (tid == 0) {
      if (s + 2 < nst) issue(s + 2);  // this stage's raw buffer has been consumed
      tc::tc_fence_after();
      const unsigned abase = tc::smem_u32(At);
      const unsigned bhi = tc::smem_u32(Bt + buf * 2 * kBT), blo = bhi + kBT;
#pragma unroll
      for (int r = 0; r < 2; ++r) {
        const unsigned dt = tmem + (unsigned)(r * N);
        const unsigned ahi = abase + (2 * r) * kAT, alo = ahi + kAT;
#pragma unroll
        for (int ks = 0; ks < T_SUB / 8; ++ks) {
          const unsigned ko = 32u * ks;
          tc::mma_tf32(dt, tc::sdesc_sw128(ahi + ko), tc::sdesc_sw128(bhi + ko), idesc,
                       s > 0 || ks > 0);
          tc::mma_tf32(dt, tc::sdesc_sw128(ahi + ko), tc::sdesc_sw128(blo + ko), idesc, true);
          tc::mma_tf32(dt, tc::sdesc_sw128(alo + ko), tc::sdesc_sw128(bhi + ko), idesc, true);
        }
      }
      tc::mma_commit(bmma);
    }
  }
  if (s_fail < 0) {
    const bool ok = tc::mbar_wait(bmma, (nst - 1) & 1);
    if (__syncthreads_or(!ok)) s_fail = nst;
  }
  if (s_fail < 0) {
    tc::tc_fence_after();
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int b = 2 * pair + r;
      if (b >= nvalid) continue;  // block-uniform
      float* g = gh + (long long)(rec0 + b) * nf * 2 * G + p0 + tid;
      for (int c0 = 0; c0 < N; c0 += 16) {
        float v[16];
        tc::tmem_ld16(tmem + ((unsigned)(warp * 32) << 16) + (unsigned)(r * N + c0), v);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int c = c0 + i;
          if (c < 2 * nf) g[(long long)c * G] += v[i];  // c = 2k + plane -> (k * 2 + plane) * G
        }
      }
    }
  } else {
    if (tid == 0) atomicExch(err, 1);
    // let this block's copies and MMAs in flight finish before leaving (bounded waits)
    const int s = s_fail;
    if (s < nst) {
      tc::mbar_wait((s & 1) ? bst1 : bst0, (s >> 1) & 1);
      if (s + 1 < nst) tc::mbar_wait(((s + 1) & 1) ? bst1 : bst0, ((s + 1) >> 1) & 1);
    }
    if (s > 0) tc::mbar_wait(bmma, (s - 1) & 1);
  }
  tc::tc_fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, ncols);
}

cudaError_t launch_dft_chunk(const float2* ring, long long slot_stride, const Layout& L,
                             int slot0, int kcount, const float* twt, int nf, int n0, int npairs,
                             int nvalid, float* gh, int rec0, int* err, cudaStream_t st) {
  if (L.G % T_P != 0 || n0 % T_SUB != 0) return cudaErrorInvalidValue;
  const size_t smem = dft_chunk_smem(nf);
  cudaError_t e =
      cudaFuncSetAttribute(k_dft_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(L.G / T_P), npairs);
  count_launches(1);
  k_dft_chunk<<<grid, T_P, smem, st>>>(ring, slot_stride, L.F, L.org, slot0, kcount, twt,
                                       n0 / T_SUB, dft_ncomp(nf), nf, L.G, gh, rec0, nvalid, err);
  return cudaGetLastError();
}

// Twiddle tiles for the tensor-core transform: for every stage of 32 levels, a hi tile and a lo
// tile of [N][32] floats in the 128-byte-swizzled K-major layout; row 2k = cos(2 pi f_k n dt),
// row 2k+1 = -sin(2 pi f_k n dt) (phase reduced as 2 pi frac(f_k n dt) in double precision),
// rows >= 2 nf and levels >= nt zero.
std::vector<float> dft_twiddle_tiles(const std::vector<double>& f, double dt, int nt) {
  const int nf = (int)f.size(), N = dft_ncomp(nf);
  const int nstg = (nt + T_SUB - 1) / T_SUB;
  std::vector<float> out((size_t)nstg * 2 * N * T_SUB, 0.f);
  for (int sg = 0; sg < nstg; ++sg) {
    unsigned char* hi = reinterpret_cast<unsigned char*>(out.data() + (size_t)sg * 2 * N * T_SUB);
    unsigned char* lo = hi + sizeof(float) * N * T_SUB;
    for (int j = 0; j < T_SUB; ++j) {
      const int n = sg * T_SUB + j;
      if (n >= nt) continue;
      for (int k = 0; k < nf; ++k) {
        double ph = f[k] * (double)n * dt;
        ph -= std::floor(ph);
        const double a = 2.0 * M_PI * ph;
        const float v[2] = {(float)std::cos(a), (float)-std::sin(a)};
        for (int q = 0; q < 2; ++q) {
          const unsigned off = tc::sw128_offset(2 * k + q, j);
          const float h = tc::tf32_hi(v[q]);
          *reinterpret_cast<float*>(hi + off) = h;
          *reinterpret_cast<float*>(lo + off) = v[q] - h;
        }
      }
    }
  }
  return out;
}

}  // namespace egh
