// Cholesky factorisation of every frequency's Hessian, Q_k = L_k L_k^H, in one launch
// (Algorithm 2 "Invert each frequency-domain matrix": the Hermitian positive-definite blocks
// are factored and kept resident instead of inverted).  One block per frequency, right-looking:
// for each column j the pivot is checked (non-positive or non-finite -> status[k] = j + 1 and the
// block stops, no trap), the column is scaled and cached in shared memory, and each warp updates
// whole rows of the trailing lower triangle with coalesced row accesses.  The upper triangle is
// zeroed at the end.
#include <cmath>

#include "egh_internal.cuh"

namespace egh {

constexpr int CH_THREADS = 512;

// piv64: the diagonal is carried in FP64 (dg[i] = Q[i][i] - sum_l |L[i][l]|^2 accumulated in
// double from the stored FP32 columns) and each pivot is taken from it, so the pivots of
// ill-conditioned matrices do not inherit the FP32 cancellation of the trailing updates; the
// off-diagonal entries stay FP32.
// Factors one n x n matrix in place with the calling block (status: 0 or failing pivot + 1).
__device__ void potrf_block(float2* __restrict__ A, int n, int* __restrict__ status_k, int piv64,
                            float2* col, double* dg, int& bad) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  __syncthreads();
  if (piv64)
    for (int i = tid; i < n; i += blockDim.x) dg[i] = (double)A[(long long)i * n + i].x;
  __syncthreads();
  for (int j = 0; j < n; ++j) {
    if (tid == 0) {
      const double d = piv64 ? dg[j] : (double)A[(long long)j * n + j].x;
      if (!(d > 0.0) || !isfinite(d)) {
        bad = j + 1;
      } else {
        const float s = piv64 ? (float)sqrt(d) : sqrtf((float)d);
        A[(long long)j * n + j] = make_float2(s, 0.f);
        col[j] = make_float2(s, 0.f);
      }
    }
    __syncthreads();
    if (bad) break;
    const float inv = 1.f / col[j].x;
    for (int i = j + 1 + tid; i < n; i += blockDim.x) {
      float2 v = A[(long long)i * n + j];
      v.x *= inv;
      v.y *= inv;
      A[(long long)i * n + j] = v;
      col[i] = v;
      if (piv64) dg[i] -= (double)v.x * v.x + (double)v.y * v.y;
    }
    __syncthreads();
    // A[i][l] -= col[i] * conj(col[l]),  j < l <= i
    for (int i = j + 1 + warp; i < n; i += nwarps) {
      const float2 ci = col[i];
      float2* rowp = A + (long long)i * n;
      for (int l = j + 1 + lane; l <= i; l += 32) {
        const float2 cl = col[l];
        float2 a = rowp[l];
        a.x -= ci.x * cl.x + ci.y * cl.y;
        a.y -= ci.y * cl.x - ci.x * cl.y;
        rowp[l] = a;
      }
    }
    __syncthreads();
  }
  if (tid == 0) *status_k = bad;
  if (!bad) {
    for (long long t = tid; t < (long long)n * n; t += blockDim.x) {
      const int i = (int)(t / n), l = (int)(t % n);
      if (l > i) A[t] = make_float2(0.f, 0.f);
    }
  }
}

__global__ void __launch_bounds__(CH_THREADS)
    k_potrf(float2* __restrict__ Lh, int n, int* __restrict__ status, int piv64) {
  extern __shared__ float2 col[];  // [n] columns, then [n] doubles of the FP64 diagonal
  double* dg = reinterpret_cast<double*>(col + n + (n & 1));
  __shared__ int bad;
  const int k = blockIdx.x;
  potrf_block(Lh + (long long)k * n * n, n, status + k, piv64, col, dg, bad);
}

// Batched form: every matrix of a list (several survey patches x all their frequencies, of
// different sizes) in one persistent launch; block b factors matrices b, b + gridDim.x, ...
template <int THREADS>
__global__ void __launch_bounds__(THREADS)
    k_potrf_many(const PotrfItem* __restrict__ items, int count, int piv64) {
  extern __shared__ float2 col[];  // sized for the largest matrix
  __shared__ int bad;
  for (int m = blockIdx.x; m < count; m += gridDim.x) {
    const PotrfItem it = items[m];
    double* dg = reinterpret_cast<double*>(col + it.n + (it.n & 1));
    potrf_block(it.A, it.n, it.status, piv64, col, dg, bad);
    __syncthreads();
  }
}

size_t potrf_smem(int nmax) {
  return sizeof(float2) * (size_t)(nmax + (nmax & 1)) + sizeof(double) * (size_t)nmax;
}

cudaError_t potrf_many_prepare(int nmax) {
  const int smem = (int)potrf_smem(nmax);
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_potrf_many<256>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  if ((e = cudaFuncSetAttribute(k_potrf_many<512>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem))) return e;
  return cudaFuncSetAttribute(k_potrf_many<1024>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

cudaError_t launch_potrf_many(const PotrfItem* items, int count, int nmax, int blocks, int threads,
                              int piv64, cudaStream_t st) {
  const size_t smem = potrf_smem(nmax);
  count_launches(1);
  switch (threads) {
    case 256: k_potrf_many<256><<<blocks, 256, smem, st>>>(items, count, piv64); break;
    case 512: k_potrf_many<512><<<blocks, 512, smem, st>>>(items, count, piv64); break;
    case 1024: k_potrf_many<1024><<<blocks, 1024, smem, st>>>(items, count, piv64); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_potrf(float2* Lh, int n, int nf, int* status, cudaStream_t st, int piv64) {
  const size_t smem = sizeof(float2) * (size_t)(n + (n & 1)) + sizeof(double) * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_potrf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_potrf<<<nf, CH_THREADS, smem, st>>>(Lh, n, status, piv64);
  return cudaGetLastError();
}

}  // namespace egh
