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

#include "egh_internal.cuh"

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
// (ring slots slot0 .. slot0+kcount-1):
//     gh[rec][k][re/im][p] += sum_j tw[n0+j][k] * u^{n0+j}[rec][p].
// A block owns D_P points of one receiver pair.  One thread streams the chunk through shared
// memory in stages of D_SUB levels with 1-D bulk (TMA) copies completing on two mbarriers
// (double buffer: the next stage lands while the current one is summed); each stage carries the
// matching twiddle rows, stored as (cos, cos, -sin, -sin) so that one 16-byte load feeds the
// packed products of both receivers.  Two threads share a pair of adjacent points, each summing
// half of the frequencies, and keep their accumulators in registers for the whole chunk; gh is
// read and written once per chunk.  Every mbarrier wait is bounded: on expiry the block records
// the error flag, waits (bounded) for its copies in flight and leaves.
// ---------------------------------------------------------------------------------------------
constexpr int D_P = 128;     // points per block
constexpr int D_SUB = 16;    // levels per stage
constexpr int D_NFH = 13;    // frequencies per thread and pass
constexpr long long kWaitLimit = 1LL << 26;  // mbarrier polls before giving up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void bulk_g2s(unsigned dst, const void* src, unsigned bytes,
                                         unsigned bar) {
  asm volatile(
      "cp.async.bulk.shared::cta.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity) {
  for (long long i = 0; i < kWaitLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

size_t dft_chunk_smem(int nf) {
  return 2 * (sizeof(float2) * D_SUB * D_P + sizeof(float4) * D_SUB * (size_t)nf);
}

__global__ void __launch_bounds__(D_P)
    k_dft_chunk(const float2* __restrict__ ring, long long slot_stride, long long pstride,
                long long org, int slot0, int kcount, const float4* __restrict__ tw4, int nf,
                int n0, long long G, float* __restrict__ gh, int rec0, int nvalid,
                int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  float2* U = reinterpret_cast<float2*>(dsm);                                    // [2][D_SUB][D_P]
  float4* T = reinterpret_cast<float4*>(dsm + sizeof(float2) * 2 * D_SUB * D_P);  // [2][D_SUB][nf]
  __shared__ __align__(8) unsigned long long bars[2];
  const int tid = threadIdx.x;
  const int pair = blockIdx.y;
  const long long p0 = (long long)blockIdx.x * D_P;
  const float2* src = ring + (long long)pair * pstride + org + p0;
  const unsigned ub0 = smem_u32(&bars[0]), ub1 = smem_u32(&bars[1]);
  if (tid == 0) {
    mbar_init(ub0, 1);
    mbar_init(ub1, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int nst = (kcount + D_SUB - 1) / D_SUB;
  const int npass = (nf + 2 * D_NFH - 1) / (2 * D_NFH);
  const int total = nst * npass;  // stages over all passes (each pass re-streams the chunk)
  auto issue = [&](int gs) {
    const int s = gs % nst, buf = gs & 1;
    const int j0 = s * D_SUB, jn = min(D_SUB, kcount - j0);
    const unsigned bar = buf ? ub1 : ub0;
    mbar_expect_tx(bar, (unsigned)(jn * D_P * sizeof(float2) + jn * nf * sizeof(float4)));
    for (int j = 0; j < jn; ++j)
      bulk_g2s(smem_u32(U + (buf * D_SUB + j) * D_P), src + (long long)(slot0 + j0 + j) * slot_stride,
               D_P * sizeof(float2), bar);
    bulk_g2s(smem_u32(T + buf * D_SUB * nf), tw4 + (long long)(n0 + j0) * nf,
             (unsigned)(jn * nf * sizeof(float4)), bar);
  };
  if (tid == 0) {
    issue(0);
    if (total > 1) issue(1);
  }
  const int fh = tid & 1, pt = tid >> 1;
  const int lp = 2 * pt;  // this thread's two points
  for (int pass = 0; pass < npass; ++pass) {
    const int fbase = pass * 2 * D_NFH + fh * D_NFH;
    const int fn = max(0, min(D_NFH, nf - fbase));
    float2 ar0[D_NFH], ai0[D_NFH], ar1[D_NFH], ai1[D_NFH];
#pragma unroll
    for (int i = 0; i < D_NFH; ++i)
      ar0[i] = ai0[i] = ar1[i] = ai1[i] = make_float2(0.f, 0.f);
    for (int s = 0; s < nst; ++s) {
      const int gs = pass * nst + s, buf = gs & 1;
      const unsigned bar = buf ? ub1 : ub0;
      const bool ok = mbar_wait_bounded(bar, (gs >> 1) & 1);
      if (__syncthreads_or(!ok)) {  // block-uniform decision: every thread leaves together
        if (tid == 0) atomicExch(err, 1);
        // let this block's copies in flight land before leaving (bounded)
        mbar_wait_bounded(bar, (gs >> 1) & 1);
        if (gs + 1 < total) mbar_wait_bounded(buf ? ub0 : ub1, ((gs + 1) >> 1) & 1);
        return;
      }
      const int jn = min(D_SUB, kcount - s * D_SUB);
      const float2* Ub = U + buf * D_SUB * D_P + lp;
      const float4* Tb = T + buf * D_SUB * nf + fbase;
      for (int j = 0; j < jn; ++j) {
        const float4 sv = *reinterpret_cast<const float4*>(Ub + j * D_P);
        const float2 s0 = make_float2(sv.x, sv.y), s1 = make_float2(sv.z, sv.w);
        const float4* tj = Tb + j * nf;
#pragma unroll
        for (int i = 0; i < D_NFH; ++i) {
          if (i < fn) {
            const float4 w = tj[i];
            const float2 c = make_float2(w.x, w.y), sn = make_float2(w.z, w.w);
            ar0[i] = __ffma2_rn(c, s0, ar0[i]);
            ai0[i] = __ffma2_rn(sn, s0, ai0[i]);
            ar1[i] = __ffma2_rn(c, s1, ar1[i]);
            ai1[i] = __ffma2_rn(sn, s1, ai1[i]);
          }
        }
      }
      __syncthreads();  // everyone is done with this buffer
      if (tid == 0 && gs + 2 < total) issue(gs + 2);
    }
    // add into gh: receiver a = lane x, receiver b = lane y of each packed accumulator
#pragma unroll
    for (int i = 0; i < D_NFH; ++i) {
      if (i < fn) {
        const int f = fbase + i;
#pragma unroll
        for (int r = 0; r < 2; ++r) {
          const int b = 2 * pair + r;
          if (b >= nvalid) continue;
          float* g = gh + ((long long)(rec0 + b) * nf + f) * 2 * G + p0 + lp;
          float2* gre = reinterpret_cast<float2*>(g);
          float2* gim = reinterpret_cast<float2*>(g + G);
          float2 re = *gre, im = *gim;
          re.x += r ? ar0[i].y : ar0[i].x;
          re.y += r ? ar1[i].y : ar1[i].x;
          im.x += r ? ai0[i].y : ai0[i].x;
          im.y += r ? ai1[i].y : ai1[i].x;
          *gre = re;
          *gim = im;
        }
      }
    }
  }
}

cudaError_t launch_dft_chunk(const float2* ring, long long slot_stride, const Layout& L,
                             int slot0, int kcount, const float4* tw4, int nf, int n0, int npairs,
                             int nvalid, float* gh, int rec0, int* err, cudaStream_t st) {
  if (L.G % D_P != 0) return cudaErrorInvalidValue;
  const size_t smem = dft_chunk_smem(nf);
  cudaError_t e =
      cudaFuncSetAttribute(k_dft_chunk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((unsigned)(L.G / D_P), npairs);
  count_launches(1);
  k_dft_chunk<<<grid, D_P, smem, st>>>(ring, slot_stride, L.F, L.org, slot0, kcount, tw4, nf, n0,
                                       L.G, gh, rec0, nvalid, err);
  return cudaGetLastError();
}

}  // namespace egh
