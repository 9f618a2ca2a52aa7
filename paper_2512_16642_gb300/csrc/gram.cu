// Per-frequency Hessians (eq. Qmatrix with S S^T replaced by its frequency-domain blocks):
//   H_k[i][j] = sum_x ghat_i(w_k, x) conj(ghat_j(w_k, x)),   Q_k = H_k + mu I.
// With M_k = [Re ghat_0; Im ghat_0; Re ghat_1; ...] (2 nrec rows, G columns) and the real
// symmetric C = M_k M_k^T:
//   Re H[i][j] = C[2i][2j] + C[2i+1][2j+1],   Im H[i][j] = C[2i+1][2j] - C[2i][2j+1].
// C is computed in 64 x 64 tiles on and above the tile diagonal only, with the grid sum split
// into `splits` ranges whose partial tiles are reduced in a second kernel (scratch workspace).
#include <cmath>

#include "egh_internal.cuh"

namespace egh {

constexpr int GT = 64;   // tile edge
constexpr int GK = 16;   // points per shared-memory stage
constexpr int GFLUSH = 128;  // stages accumulated before adding into the running total

__host__ __device__ int gram_tiles(int nrec) { return (2 * nrec + GT - 1) / GT; }

size_t gram_workspace_floats(int nrec, int nf, int splits) {
  const int nt = gram_tiles(nrec);
  const size_t pairs = (size_t)nt * (nt + 1) / 2;
  return (size_t)splits * nf * pairs * GT * GT;
}

__device__ inline const float* m_row(const float* gh, int a, int k, int nf, long long G) {
  return gh + ((long long)((a >> 1) * nf + k) * 2 + (a & 1)) * G;
}

__global__ void __launch_bounds__(256)
    k_gram_partial(const float* __restrict__ gh, int nrec, int nf, long long G, int ntile,
                   long long split_len, float* __restrict__ part) {
  __shared__ __align__(16) float As[GK][GT + 4];
  __shared__ __align__(16) float Bs[GK][GT + 4];
  const int pair = blockIdx.x, k = blockIdx.y, s = blockIdx.z;
  int ta = 0, rem = pair;
  while (rem >= ntile - ta) {
    rem -= ntile - ta;
    ++ta;
  }
  const int tb = ta + rem;
  const int rows = 2 * nrec;
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int lr = tid >> 2, lp = (tid & 3) * 4;
  const int ra = ta * GT + lr, rb = tb * GT + lr;
  const float* arow = ra < rows ? m_row(gh, ra, k, nf, G) : nullptr;
  const float* brow = rb < rows ? m_row(gh, rb, k, nf, G) : nullptr;
  const long long p0 = (long long)s * split_len;
  const long long p1 = min(G, p0 + split_len);

  float acc[4][4], tot[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = tot[i][j] = 0.f;
  int stages = 0;
  for (long long p = p0; p < p1; p += GK) {
    float4 va = make_float4(0.f, 0.f, 0.f, 0.f), vb = va;
    if (arow) va = *reinterpret_cast<const float4*>(arow + p + lp);
    if (brow) vb = *reinterpret_cast<const float4*>(brow + p + lp);
    As[lp + 0][lr] = va.x;
    As[lp + 1][lr] = va.y;
    As[lp + 2][lr] = va.z;
    As[lp + 3][lr] = va.w;
    Bs[lp + 0][lr] = vb.x;
    Bs[lp + 1][lr] = vb.y;
    Bs[lp + 2][lr] = vb.z;
    Bs[lp + 3][lr] = vb.w;
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      const float4 a4 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w};
      const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (++stages == GFLUSH) {
      stages = 0;
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          tot[i][j] += acc[i][j];
          acc[i][j] = 0.f;
        }
    }
  }
  const int npairs = ntile * (ntile + 1) / 2;
  float* out = part + (((long long)s * nf + k) * npairs + pair) * (GT * GT);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float4 v;
    v.x = tot[i][0] + acc[i][0];
    v.y = tot[i][1] + acc[i][1];
    v.z = tot[i][2] + acc[i][2];
    v.w = tot[i][3] + acc[i][3];
    *reinterpret_cast<float4*>(out + (ty * 4 + i) * GT + tx * 4) = v;
  }
}

cudaError_t launch_gram_partial(const float* gh, int nrec, int nf, long long G, int splits,
                                float* part, cudaStream_t st) {
  const int nt = gram_tiles(nrec);
  const int npairs = nt * (nt + 1) / 2;
  long long split_len = (G + splits - 1) / splits;
  split_len = (split_len + GK - 1) / GK * GK;
  dim3 grid(npairs, nf, splits);
  count_launches(1);
  k_gram_partial<<<grid, 256, 0, st>>>(gh, nrec, nf, G, nt, split_len, part);
  return cudaGetLastError();
}

// C[a][b] summed over splits, read from the tile pair with ta <= tb (C is symmetric).
__device__ inline float c_entry(const float* part, int a, int b, int k, int nf, int ntile,
                                int npairs, int splits) {
  if (a / GT > b / GT) {
    const int t = a;
    a = b;
    b = t;
  }
  const int ta = a / GT, tb = b / GT;
  const int pair = ta * ntile - ta * (ta - 1) / 2 + (tb - ta);
  const long long off = (long long)(a % GT) * GT + (b % GT);
  double sum = 0.0;
  for (int s = 0; s < splits; ++s)
    sum += part[(((long long)s * nf + k) * npairs + pair) * (GT * GT) + off];
  return (float)sum;
}

__global__ void k_gram_finish(const float* __restrict__ part, int nrec, int nf, int splits,
                              float2* __restrict__ Qh) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  const int i = blockIdx.y;
  const int k = blockIdx.z;
  if (j >= nrec) return;
  const int ntile = gram_tiles(nrec);
  const int npairs = ntile * (ntile + 1) / 2;
  const int a = min(i, j), b = max(i, j);
  const float rr = c_entry(part, 2 * a, 2 * b, k, nf, ntile, npairs, splits);
  const float ii = c_entry(part, 2 * a + 1, 2 * b + 1, k, nf, ntile, npairs, splits);
  float im = 0.f;
  if (a != b)
    im = c_entry(part, 2 * a + 1, 2 * b, k, nf, ntile, npairs, splits) -
         c_entry(part, 2 * a, 2 * b + 1, k, nf, ntile, npairs, splits);
  // entry (a, b) with a <= b; (b, a) is its conjugate
  Qh[((long long)k * nrec + i) * nrec + j] = make_float2(rr + ii, i <= j ? im : -im);
}

cudaError_t launch_gram_finish(const float* part, int nrec, int nf, int splits, float2* Qh,
                               cudaStream_t st) {
  dim3 grid((nrec + 127) / 128, nrec, nf);
  count_launches(1);
  k_gram_finish<<<grid, 128, 0, st>>>(part, nrec, nf, splits, Qh);
  return cudaGetLastError();
}

// d_sum[0] = sum over k, i of Re Qh[k][i][i]   (one block)
__global__ void k_diag_sum(const float2* __restrict__ Qh, int nrec, int nf, double* d_sum) {
  __shared__ double red[256];
  double s = 0.0;
  for (int t = threadIdx.x; t < nrec * nf; t += blockDim.x) {
    const int k = t / nrec, i = t % nrec;
    s += (double)Qh[((long long)k * nrec + i) * nrec + i].x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d_sum[0] = red[0];
}

cudaError_t launch_diag_sum(const float2* Qh, int nrec, int nf, double* d_sum, cudaStream_t st) {
  count_launches(1);
  k_diag_sum<<<1, 256, 0, st>>>(Qh, nrec, nf, d_sum);
  return cudaGetLastError();
}

// ||Q_k||_F^2 per frequency: one block per frequency, FP32 squares summed in FP64.
__global__ void k_fro2(const float2* __restrict__ Qh, int n, double* d_out) {
  __shared__ double red[256];
  const long long n2 = (long long)n * n;
  const float2* A = Qh + (long long)blockIdx.x * n2;
  double s = 0.0;
  for (long long t = threadIdx.x; t < n2; t += blockDim.x) {
    const float2 a = A[t];
    s += (double)a.x * a.x + (double)a.y * a.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) d_out[blockIdx.x] = red[0];
}

cudaError_t launch_fro2(const float2* Qh, int n, int nf, double* d_out, cudaStream_t st) {
  count_launches(1);
  k_fro2<<<nf, 256, 0, st>>>(Qh, n, d_out);
  return cudaGetLastError();
}

// Largest eigenvalue of Q_k^{-1} = W_k^H W_k (W = L^{-1}, lower triangular) by 40 steps of
// power iteration in FP32, one block per frequency: lam[k] = ||W^H W v|| / ||v|| for the last v.
// It approaches 1 / lambda_min(Q_k) from below.
__global__ void k_inv_power(const float2* __restrict__ Wh, int n, double* lam) {
  extern __shared__ float2 pv[];  // v [n], y [n]
  __shared__ float red[256];
  float2* v = pv;
  float2* y = pv + n;
  const float2* W = Wh + (long long)blockIdx.x * n * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = make_float2(1.f + 0.01f * (i % 7), 0.f);
  __syncthreads();
  float norm = 0.f;
  auto reduce = [&](float x) {
    red[threadIdx.x] = x;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    const float r = red[0];
    __syncthreads();
    return r;
  };
  float vv = reduce([&] {
    float a = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) a += v[i].x * v[i].x + v[i].y * v[i].y;
    return a;
  }());
  for (int it = 0; it < 40; ++it) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // y = W v
      float re = 0.f, im = 0.f;
      for (int j = 0; j <= i; ++j) {
        const float2 a = W[(long long)i * n + j], b = v[j];
        re = fmaf(a.x, b.x, fmaf(-a.y, b.y, re));
        im = fmaf(a.x, b.y, fmaf(a.y, b.x, im));
      }
      y[i] = make_float2(re, im);
    }
    __syncthreads();
    float a2 = 0.f;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {  // v' = W^H y
      float re = 0.f, im = 0.f;
      for (int j = i; j < n; ++j) {
        const float2 a = W[(long long)j * n + i], b = y[j];
        re = fmaf(a.x, b.x, fmaf(a.y, b.y, re));
        im = fmaf(a.x, b.y, fmaf(-a.y, b.x, im));
      }
      v[i] = make_float2(re, im);
      a2 += re * re + im * im;
    }
    __syncthreads();
    const float w2 = reduce(a2);
    norm = sqrtf(w2 / vv);
    const float sc = 1.f / sqrtf(w2);
    for (int i = threadIdx.x; i < n; i += blockDim.x) v[i] = make_float2(v[i].x * sc, v[i].y * sc);
    vv = 1.f;
    __syncthreads();
  }
  if (threadIdx.x == 0) lam[blockIdx.x] = norm;
}

cudaError_t launch_inv_power(const float2* Wh, int n, int nf, double* lam, cudaStream_t st) {
  const size_t smem = sizeof(float2) * 2 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_inv_power, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_inv_power<<<nf, 256, smem, st>>>(Wh, n, lam);
  return cudaGetLastError();
}

// Largest eigenvalue of each Hermitian H_k by power iteration (fixed 300 iterations, Rayleigh
// quotient), one block per frequency; d_lmax[k].
constexpr int PI_ITERS = 300;

__global__ void k_lambda_max(const float2* __restrict__ Qh, int n, double* d_lmax) {
  extern __shared__ double sv[];  // v: 2n doubles, y: 2n doubles
  __shared__ double red[256];
  const int k = blockIdx.x;
  const float2* A = Qh + (long long)k * n * n;
  double* v = sv;
  double* y = sv + 2 * n;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    v[2 * i] = 1.0 + 0.01 * (i % 7);
    v[2 * i + 1] = 0.0;
  }
  __syncthreads();
  double lam = 0.0;
  for (int it = 0; it < PI_ITERS; ++it) {
    // y = A v
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      double re = 0.0, im = 0.0;
      for (int j = 0; j < n; ++j) {
        const float2 a = A[(long long)i * n + j];
        re += a.x * v[2 * j] - a.y * v[2 * j + 1];
        im += a.x * v[2 * j + 1] + a.y * v[2 * j];
      }
      y[2 * i] = re;
      y[2 * i + 1] = im;
    }
    __syncthreads();
    // Rayleigh quotient v^H y / v^H v and the norm of y
    double num = 0.0, den = 0.0, yy = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      num += v[2 * i] * y[2 * i] + v[2 * i + 1] * y[2 * i + 1];
      den += v[2 * i] * v[2 * i] + v[2 * i + 1] * v[2 * i + 1];
      yy += y[2 * i] * y[2 * i] + y[2 * i + 1] * y[2 * i + 1];
    }
    double vals[3] = {num, den, yy};
    for (int q = 0; q < 3; ++q) {
      red[threadIdx.x] = vals[q];
      __syncthreads();
      for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
        __syncthreads();
      }
      vals[q] = red[0];
      __syncthreads();
    }
    lam = vals[1] > 0.0 ? vals[0] / vals[1] : 0.0;
    const double inv = vals[2] > 0.0 ? 1.0 / sqrt(vals[2]) : 0.0;
    for (int i = threadIdx.x; i < 2 * n; i += blockDim.x) v[i] = y[i] * inv;
    __syncthreads();
  }
  if (threadIdx.x == 0) d_lmax[k] = lam;
}

cudaError_t launch_lambda_max(const float2* Qh, int nrec, int nf, double* d_lmax,
                              cudaStream_t st) {
  const size_t smem = sizeof(double) * 4 * (size_t)nrec;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_lambda_max, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_lambda_max<<<nf, 256, smem, st>>>(Qh, nrec, d_lmax);
  return cudaGetLastError();
}

// Qh += mu I; Lh = Qh.
__global__ void k_add_mu_copy(float2* __restrict__ Qh, float2* __restrict__ Lh, long long n2,
                              int nrec, float mu) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2;
       t += (long long)gridDim.x * blockDim.x) {
    const long long local = t % ((long long)nrec * nrec);
    float2 v = Qh[t];
    if (local / nrec == local % nrec) {
      v.x += mu;
      Qh[t] = v;
    }
    Lh[t] = v;
  }
}

cudaError_t launch_add_mu_copy(float2* Qh, float2* Lh, int nrec, int nf, float mu,
                               cudaStream_t st) {
  const long long n2 = (long long)nf * nrec * nrec;
  long long blocks = (n2 + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launches(1);
  k_add_mu_copy<<<(int)blocks, 256, 0, st>>>(Qh, Lh, n2, nrec, mu);
  return cudaGetLastError();
}

// The penalty of the Hessians changed from mu_old to mu_new: Qh's diagonal has mu_old removed
// (when nonzero) and mu_new added, and Lh = Qh.  From mu_old = 0 the result is the one of
// launch_add_mu_copy with mu_new, bit for bit.
__global__ void k_set_mu_copy(float2* __restrict__ Qh, float2* __restrict__ Lh, long long n2,
                              int nrec, float mu_old, float mu_new) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n2;
       t += (long long)gridDim.x * blockDim.x) {
    const long long local = t % ((long long)nrec * nrec);
    float2 v = Qh[t];
    if (local / nrec == local % nrec) {
      if (mu_old != 0.f) v.x -= mu_old;
      v.x += mu_new;
      Qh[t] = v;
    }
    Lh[t] = v;
  }
}

cudaError_t launch_add_mu_copy_delta(float2* Qh, float2* Lh, int nrec, int nf, double mu_old,
                                     double mu_new, cudaStream_t st) {
  const long long n2 = (long long)nf * nrec * nrec;
  long long blocks = (n2 + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launches(1);
  k_set_mu_copy<<<(int)blocks, 256, 0, st>>>(Qh, Lh, n2, nrec, (float)mu_old, (float)mu_new);
  return cudaGetLastError();
}

}  // namespace egh
