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
// One leapfrog step for a batch of receivers.  Each warp owns 32 columns and marches down TZ rows,
// keeping the nine z-neighbours of its column in registers; the x-neighbours come from a
// 40-float row staged in shared memory (32 + 4 halo on each side).  Reads of guard rows and
// padding columns return the zero boundary, so there is no bounds test on loads.
// ---------------------------------------------------------------------------------------------
constexpr int FD_WARPS = 4;
constexpr int FD_TZ = 32;

__global__ void __launch_bounds__(32 * FD_WARPS)
    k_fd_step(const float* __restrict__ ucur, const float* __restrict__ uprev,
              float* __restrict__ unext, const float* __restrict__ c1,
              const float* __restrict__ c3, int NZ, int NX, int PX, long long org,
              long long fstride, Stencil S) {
  __shared__ float srow[FD_WARPS][40];
  const int lane = threadIdx.x;
  const int w = threadIdx.y;
  const int x0 = blockIdx.x * 32;
  const int x = x0 + lane;
  const int z0 = (blockIdx.y * FD_WARPS + w) * FD_TZ;
  if (z0 >= NZ) return;  // whole warp leaves; only warp-level synchronisation below
  const long long boff = (long long)blockIdx.z * fstride + org;
  const float* __restrict__ uc = ucur + boff;
  const float* __restrict__ up = uprev + boff;
  float* __restrict__ un = unext + boff;
  const float* __restrict__ k1 = c1 + org;
  const float* __restrict__ k3 = c3 + org;
  float* row = srow[w];

  float q[9];
#pragma unroll
  for (int i = 0; i < 8; ++i) q[i + 1] = uc[(long long)(z0 - 4 + i) * PX + x];
  const int zend = min(z0 + FD_TZ, NZ);
  for (int z = z0; z < zend; ++z) {
#pragma unroll
    for (int i = 0; i < 8; ++i) q[i] = q[i + 1];
    const long long rz = (long long)z * PX;
    q[8] = uc[rz + (long long)4 * PX + x];
    row[lane + 4] = q[4];
    if (lane < 4) {
      row[lane] = uc[rz + x0 - 4 + lane];
    } else if (lane >= 28) {
      row[lane + 8] = uc[rz + x0 + 4 + lane];
    }
    __syncwarp();
    if (x < NX) {
      float lap = S.c0 * q[4];
      lap = fmaf(S.cz[0], q[3] + q[5], lap);
      lap = fmaf(S.cz[1], q[2] + q[6], lap);
      lap = fmaf(S.cz[2], q[1] + q[7], lap);
      lap = fmaf(S.cz[3], q[0] + q[8], lap);
      lap = fmaf(S.cx[0], row[lane + 3] + row[lane + 5], lap);
      lap = fmaf(S.cx[1], row[lane + 2] + row[lane + 6], lap);
      lap = fmaf(S.cx[2], row[lane + 1] + row[lane + 7], lap);
      lap = fmaf(S.cx[3], row[lane + 0] + row[lane + 8], lap);
      const long long p = rz + x;
      const float uo = up[p];
      un[p] = fmaf(k3[p], lap, fmaf(k1[p], q[4] - uo, uo));
    }
    __syncwarp();
  }
}

cudaError_t launch_fd_step(const float* ucur, const float* uprev, float* unext, const float* c1,
                           const float* c3, const Layout& L, const Stencil& S, int nb,
                           long long fstride, cudaStream_t st) {
  dim3 block(32, FD_WARPS);
  dim3 grid(L.PX / 32, (L.NZ + FD_WARPS * FD_TZ - 1) / (FD_WARPS * FD_TZ), nb);
  count_launches(1);
  k_fd_step<<<grid, block, 0, st>>>(ucur, uprev, unext, c1, c3, L.NZ, L.NX, L.PX, L.org, fstride,
                                    S);
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
// Each thread owns two adjacent points; the chunk's twiddles sit in shared memory.
// ---------------------------------------------------------------------------------------------
template <int K>
__global__ void __launch_bounds__(256)
    k_dft_chunk(const float* __restrict__ ring, long long slot_stride, long long fstride,
                long long org, const float2* __restrict__ tw, int nf, int n0, int kcount,
                long long G, float* __restrict__ gh, int rec0) {
  extern __shared__ float2 stw[];  // [K][nf]
  for (int i = threadIdx.x; i < K * nf; i += blockDim.x)
    stw[i] = (i < kcount * nf) ? tw[(long long)n0 * nf + i] : make_float2(0.f, 0.f);
  __syncthreads();
  const int b = blockIdx.y;
  const long long p = 2 * ((long long)blockIdx.x * blockDim.x + threadIdx.x);
  if (p >= G) return;
  const float* src = ring + (long long)b * fstride + org + p;
  float2 s[K];
#pragma unroll
  for (int j = 0; j < K; ++j)
    s[j] = (j < kcount) ? *reinterpret_cast<const float2*>(src + j * slot_stride)
                        : make_float2(0.f, 0.f);
  float* g = gh + (long long)(rec0 + b) * nf * 2 * G + p;
  for (int k = 0; k < nf; ++k) {
    float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const float2 w = stw[j * nf + k];
      ar0 = fmaf(w.x, s[j].x, ar0);
      ai0 = fmaf(w.y, s[j].x, ai0);
      ar1 = fmaf(w.x, s[j].y, ar1);
      ai1 = fmaf(w.y, s[j].y, ai1);
    }
    float2* gre = reinterpret_cast<float2*>(g + (long long)k * 2 * G);
    float2* gim = reinterpret_cast<float2*>(g + (long long)k * 2 * G + G);
    float2 r = *gre;
    r.x += ar0;
    r.y += ar1;
    *gre = r;
    float2 m = *gim;
    m.x += ai0;
    m.y += ai1;
    *gim = m;
  }
}

cudaError_t launch_dft_chunk(const float* ring, long long slot_stride, long long fstride,
                             const Layout& L, const float2* tw, int nf, int n0, int kcount, int K,
                             int nb, float* gh, int rec0, cudaStream_t st) {
  const long long threads = L.G / 2;
  dim3 grid((unsigned)((threads + 255) / 256), nb);
  const size_t smem = sizeof(float2) * (size_t)K * nf;
  switch (K) {
    case 16:
      count_launches(1);
      k_dft_chunk<16><<<grid, 256, smem, st>>>(ring, slot_stride, fstride, L.org, tw, nf, n0,
                                               kcount, L.G, gh, rec0);
      break;
    case 32:
      count_launches(1);
      k_dft_chunk<32><<<grid, 256, smem, st>>>(ring, slot_stride, fstride, L.org, tw, nf, n0,
                                               kcount, L.G, gh, rec0);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

}  // namespace egh
