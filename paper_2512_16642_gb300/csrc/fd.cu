// Time-domain finite differences for the receiver-side Green functions and their on-the-fly
// transform at the Nf frequencies (Section "Direct Hessian-inverse computation": one wave-equation
// solve per receiver with a Dirac source at the receiver; eq. wave_eq).
//
// Scheme (the paper does not give one): second-order leapfrog, eighth-order Laplacian, damping
// written symmetrically so that reciprocity holds,
//     u^{n+1} = c1 (u^n - u^{n-1}) + u^{n-1} + c3 L u^n,   c1 = 2/(1+a), c3 = dt^2 v^2/(1+a),
// a = eta dt / 2 (from (1+a) u^{n+1} = 2 u^n - (1-a) u^{n-1} + dt^2 v^2 L u^n, since
// (1-a)/(1+a) = c1 - 1).
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
// Coefficients on the padded, pitched grid.  Velocity is extended into the sponge by edge
// replication; eta = eta0 (d/L)^2 per axis, eta0 = 1.5 vmax ln(1/R) / L.
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
                             float* __restrict__ c1, float* __restrict__ c3) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int z = blockIdx.y;
  if (x >= L.PX || z >= L.NZ) return;
  const long long p = L.org + (long long)z * L.PX + x;
  if (x >= L.NX) {
    c1[p] = 0.f;
    c3[p] = 0.f;
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
  c1[p] = (float)(2.0 / (1.0 + a));
  c3[p] = (float)(dt * dt * v * v / (1.0 + a));
}

cudaError_t launch_build_coef(const float* vel, const Layout& L, double dz, double dx, double dt,
                              double R, const float* d_vmax, float* c1, float* c3,
                              cudaStream_t st) {
  dim3 grid((L.PX + 127) / 128, L.NZ);
  count_launches(1);
  k_build_coef<<<grid, 128, 0, st>>>(vel, L, dz, dx, dt, R, d_vmax, c1, c3);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// One leapfrog step for a batch of receivers.  Each warp owns 32 columns and marches down FD_TZ
// rows for RB receivers at once (the coefficients of a point are loaded once for all of them),
// keeping the nine z-neighbours of its column in registers; the x-neighbours come from a
// 40-float row staged in shared memory (32 + 4 halo on each side).  Rows are processed in groups
// of FD_U whose loads are all issued before the group is computed, so that many independent
// loads are in flight per warp.  Reads of guard rows and padding columns return the zero
// boundary, so there is no bounds test on loads; rows past the warp's range are not loaded.
// ---------------------------------------------------------------------------------------------
constexpr int FD_WARPS = 4;
constexpr int FD_TZ = 16;
constexpr int FD_U = 4;

template <int RB>
__global__ void __launch_bounds__(32 * FD_WARPS)
    k_fd_step(const float* __restrict__ ucur, const float* __restrict__ uprev,
              float* __restrict__ unext, const float* __restrict__ c1,
              const float* __restrict__ c3, int NZ, int NX, int PX, long long org,
              long long fstride, Stencil S, int nb) {
  __shared__ float srow[FD_WARPS][RB][40];
  const int lane = threadIdx.x;
  const int w = threadIdx.y;
  const int x0 = blockIdx.x * 32;
  const int x = x0 + lane;
  const int z0 = (blockIdx.y * FD_WARPS + w) * FD_TZ;
  if (z0 >= NZ) return;  // whole warp leaves; only warp-level synchronisation below
  const int b0 = blockIdx.z * RB;
  const float* uc[RB];
  const float* up[RB];
  float* un[RB];
#pragma unroll
  for (int r = 0; r < RB; ++r) {
    // a partial last group repeats its last receiver (same values written twice)
    const long long boff = (long long)min(b0 + r, nb - 1) * fstride + org;
    uc[r] = ucur + boff;
    up[r] = uprev + boff;
    un[r] = unext + boff;
  }
  const float* __restrict__ k1 = c1 + org;
  const float* __restrict__ k3 = c3 + org;
  const bool halo = lane < 4 || lane >= 28;
  const int hcol = lane < 4 ? x0 - 4 + lane : x0 + 4 + lane;
  const int hslot = lane < 4 ? lane : lane + 8;

  float q[RB][9];
#pragma unroll
  for (int r = 0; r < RB; ++r)
#pragma unroll
    for (int i = 0; i < 8; ++i) q[r][i + 1] = uc[r][(long long)(z0 - 4 + i) * PX + x];
  const int zend = min(z0 + FD_TZ, NZ);
  for (int zg = z0; zg < zend; zg += FD_U) {
    float qn[RB][FD_U], hv[RB][FD_U], uo[RB][FD_U], a1[FD_U], a3[FD_U];
#pragma unroll
    for (int i = 0; i < FD_U; ++i) {
      if (zg + i < zend) {
        const long long rz = (long long)(zg + i) * PX;
        a1[i] = k1[rz + x];
        a3[i] = k3[rz + x];
#pragma unroll
        for (int r = 0; r < RB; ++r) {
          qn[r][i] = uc[r][rz + (long long)4 * PX + x];
          uo[r][i] = up[r][rz + x];
          hv[r][i] = halo ? uc[r][rz + hcol] : 0.f;
        }
      }
    }
#pragma unroll
    for (int i = 0; i < FD_U; ++i) {
      if (zg + i < zend) {
        const long long p = (long long)(zg + i) * PX + x;
#pragma unroll
        for (int r = 0; r < RB; ++r) {
#pragma unroll
          for (int j = 0; j < 8; ++j) q[r][j] = q[r][j + 1];
          q[r][8] = qn[r][i];
          srow[w][r][lane + 4] = q[r][4];
          if (halo) srow[w][r][hslot] = hv[r][i];
        }
        __syncwarp();
        if (x < NX) {
#pragma unroll
          for (int r = 0; r < RB; ++r) {
            // Laplacian as sum_k c_k [(u_{+k} - u) + (u_{-k} - u)] (c_0 = -2 sum_k c_k):
            // neighbour differences of a well-sampled field are exact in float32, so the large
            // cancelling terms of c_0 u + sum_k c_k (u_{+k} + u_{-k}) never form.
            const float* row = srow[w][r];
            const float u0 = q[r][4];
            float lap = S.cz[0] * ((q[r][3] - u0) + (q[r][5] - u0));
            lap = fmaf(S.cz[1], (q[r][2] - u0) + (q[r][6] - u0), lap);
            lap = fmaf(S.cz[2], (q[r][1] - u0) + (q[r][7] - u0), lap);
            lap = fmaf(S.cz[3], (q[r][0] - u0) + (q[r][8] - u0), lap);
            lap = fmaf(S.cx[0], (row[lane + 3] - u0) + (row[lane + 5] - u0), lap);
            lap = fmaf(S.cx[1], (row[lane + 2] - u0) + (row[lane + 6] - u0), lap);
            lap = fmaf(S.cx[2], (row[lane + 1] - u0) + (row[lane + 7] - u0), lap);
            lap = fmaf(S.cx[3], (row[lane + 0] - u0) + (row[lane + 8] - u0), lap);
            un[r][p] = fmaf(a3[i], lap, fmaf(a1[i], u0 - uo[r][i], uo[r][i]));
          }
        }
        __syncwarp();
      }
    }
  }
}

cudaError_t launch_fd_step(const float* ucur, const float* uprev, float* unext, const float* c1,
                           const float* c3, const Layout& L, const Stencil& S, int nb,
                           long long fstride, cudaStream_t st) {
  dim3 block(32, FD_WARPS);
  const int rows = (L.NZ + FD_WARPS * FD_TZ - 1) / (FD_WARPS * FD_TZ);
  if (nb >= 2) {
    dim3 grid(L.PX / 32, rows, (nb + 1) / 2);
    count_launches(1);
    k_fd_step<2><<<grid, block, 0, st>>>(ucur, uprev, unext, c1, c3, L.NZ, L.NX, L.PX, L.org,
                                         fstride, S, nb);
  } else {
    dim3 grid(L.PX / 32, rows, nb);
    count_launches(1);
    k_fd_step<1><<<grid, block, 0, st>>>(ucur, uprev, unext, c1, c3, L.NZ, L.NX, L.PX, L.org,
                                         fstride, S, nb);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Point sources: u[b][pts[b]] += c3[pts[b]] * amp * scale  (source term dt^2 v^2 f^n / (1 + a),
// f^n = amp / (dx dz)).  amp comes from amp_dev[b] when given, else amp_host.
// ---------------------------------------------------------------------------------------------
__global__ void k_inject(float* __restrict__ u, long long fstride, const int* __restrict__ pts,
                         const float* __restrict__ c3, int nb, const float* __restrict__ amp_dev,
                         float amp_host, float scale) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= nb) return;
  const int p = pts[b];
  const float a = amp_dev ? amp_dev[b] : amp_host;
  u[(long long)b * fstride + p] += c3[p] * a * scale;
}

cudaError_t launch_inject(float* u, long long fstride, const int* pts, const float* c3, int nb,
                          const float* amp_dev, float amp_host, float scale, cudaStream_t st) {
  count_launches(1);
  k_inject<<<(nb + 127) / 128, 128, 0, st>>>(u, fstride, pts, c3, nb, amp_dev, amp_host, scale);
  return cudaGetLastError();
}

// traces[b][r][t] = u[b][rec_pts[r]]   (rec_pts are offsets inside a level)
__global__ void k_record(const float* __restrict__ u, long long fstride,
                         const int* __restrict__ rec_pts, int nrec, int nb,
                         float* __restrict__ traces, int nt, int t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nrec * nb) return;
  const int b = i / nrec, r = i % nrec;
  traces[((long long)b * nrec + r) * nt + t] = u[(long long)b * fstride + rec_pts[r]];
}

cudaError_t launch_record(const float* u, long long fstride, const int* rec_pts, int nrec, int nb,
                          float* traces, int nt, int t, cudaStream_t st) {
  const int n = nrec * nb;
  count_launches(1);
  k_record<<<(n + 255) / 256, 256, 0, st>>>(u, fstride, rec_pts, nrec, nb, traces, nt, t);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// On-the-fly transform, one chunk of kcount <= K consecutive levels n0 .. n0+kcount-1 (ring slots
// 0 .. kcount-1):  gh[rec0+b][k][re/im][p] += sum_j tw[n0+j][k] * u^{n0+j}[b][p].
// A block owns DT_P points of one receiver.  One thread stages the chunk's rows of those points
// into shared memory with 1-D bulk (TMA) copies completing on an mbarrier; the chunk's twiddles
// are staged alongside.  Each thread then owns two adjacent points and keeps the accumulators of
// DT_NF frequencies in registers (several passes when nf > DT_NF), adding them into gh once per
// chunk.  The mbarrier wait is bounded: on expiry the block records an error flag and leaves.
// ---------------------------------------------------------------------------------------------
constexpr int DT_P = 256;       // points per block
constexpr int DT_THREADS = 128; // two points per thread
constexpr int DT_NF = 26;       // frequencies per register pass
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

template <int K>
__global__ void __launch_bounds__(DT_THREADS)
    k_dft_chunk(const float* __restrict__ ring, long long slot_stride, long long fstride,
                long long org, const float2* __restrict__ tw, int nf, int n0, int kcount,
                long long G, float* __restrict__ gh, int rec0, int* __restrict__ err) {
  extern __shared__ __align__(128) unsigned char dsm[];
  float* U = reinterpret_cast<float*>(dsm);                      // [K][DT_P]
  float2* T = reinterpret_cast<float2*>(dsm + sizeof(float) * K * DT_P);  // [K][nf]
  __shared__ __align__(8) unsigned long long bar;
  const int tid = threadIdx.x;
  const int b = blockIdx.y;
  const long long p0 = (long long)blockIdx.x * DT_P;
  const unsigned ubar = smem_u32(&bar);
  if (tid == 0) {
    mbar_init(ubar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (tid == 0) {
    mbar_expect_tx(ubar, (unsigned)(kcount * DT_P * sizeof(float)));
    const float* src = ring + (long long)b * fstride + org + p0;
    for (int j = 0; j < kcount; ++j)
      bulk_g2s(smem_u32(U + j * DT_P), src + j * slot_stride, DT_P * sizeof(float), ubar);
  }
  for (int i = tid; i < kcount * nf; i += DT_THREADS) T[i] = tw[(long long)n0 * nf + i];
  long long polls = 0;
  while (!mbar_try_wait(ubar, 0)) {
    if (++polls > kWaitLimit) {
      atomicExch(err, 1);
      break;
    }
  }
  __syncthreads();
  if (polls > kWaitLimit) {
    // copies may still be landing in shared memory; wait for them (bounded) before leaving
    for (long long i = 0; i < kWaitLimit && !mbar_try_wait(ubar, 0); ++i) {
    }
    return;
  }
  const int lp = 2 * tid;
  float* g = gh + (long long)(rec0 + b) * nf * 2 * G + p0 + lp;
  for (int f0 = 0; f0 < nf; f0 += DT_NF) {
    const int fn = min(DT_NF, nf - f0);
    float ar[DT_NF][2], ai[DT_NF][2];
#pragma unroll
    for (int f = 0; f < DT_NF; ++f) ar[f][0] = ar[f][1] = ai[f][0] = ai[f][1] = 0.f;
#pragma unroll 4
    for (int j = 0; j < kcount; ++j) {
      const float2 s = *reinterpret_cast<const float2*>(U + j * DT_P + lp);
      const float2* tj = T + j * nf + f0;
#pragma unroll
      for (int f = 0; f < DT_NF; ++f) {
        if (f < fn) {
          const float2 w = tj[f];
          ar[f][0] = fmaf(w.x, s.x, ar[f][0]);
          ai[f][0] = fmaf(w.y, s.x, ai[f][0]);
          ar[f][1] = fmaf(w.x, s.y, ar[f][1]);
          ai[f][1] = fmaf(w.y, s.y, ai[f][1]);
        }
      }
    }
#pragma unroll
    for (int f = 0; f < DT_NF; ++f) {
      if (f < fn) {
        float2* gre = reinterpret_cast<float2*>(g + (long long)(f0 + f) * 2 * G);
        float2* gim = reinterpret_cast<float2*>(g + (long long)(f0 + f) * 2 * G + G);
        float2 r = *gre;
        r.x += ar[f][0];
        r.y += ar[f][1];
        *gre = r;
        float2 m = *gim;
        m.x += ai[f][0];
        m.y += ai[f][1];
        *gim = m;
      }
    }
  }
}

size_t dft_chunk_smem(int K, int nf) {
  return sizeof(float) * (size_t)K * DT_P + sizeof(float2) * (size_t)K * nf;
}

cudaError_t launch_dft_chunk(const float* ring, long long slot_stride, long long fstride,
                             const Layout& L, const float2* tw, int nf, int n0, int kcount, int K,
                             int nb, float* gh, int rec0, int* err, cudaStream_t st) {
  if (L.G % DT_P != 0) return cudaErrorInvalidValue;
  dim3 grid((unsigned)(L.G / DT_P), nb);
  const size_t smem = dft_chunk_smem(K, nf);
  cudaError_t e = cudaSuccess;
  switch (K) {
    case 32:
      e = cudaFuncSetAttribute(k_dft_chunk<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      count_launches(1);
      k_dft_chunk<32><<<grid, DT_THREADS, smem, st>>>(ring, slot_stride, fstride, L.org, tw, nf,
                                                      n0, kcount, L.G, gh, rec0, err);
      break;
    case 64:
      e = cudaFuncSetAttribute(k_dft_chunk<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)smem);
      if (e != cudaSuccess) return e;
      count_launches(1);
      k_dft_chunk<64><<<grid, DT_THREADS, smem, st>>>(ring, slot_stride, fstride, L.org, tw, nf,
                                                      n0, kcount, L.G, gh, rec0, err);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace egh
