// Cholesky factorisation of every frequency's Hessian, Q_k = L_k L_k^H, in one launch
// (Algorithm 2 inverts each frequency's matrix; here the Hermitian positive-definite blocks
// are factored and kept resident instead).  One block per frequency, right-looking:
// for each column j the pivot is checked (non-positive or non-finite -> status[k] = j + 1 and the
// block stops, no trap), the column is scaled and cached in shared memory, and each warp updates
// whole rows of the trailing lower triangle with coalesced row accesses.  The upper triangle is
// zeroed at the end.
#include <algorithm>
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

// Blocked form (matrices whose 32-column panel fits in shared memory): the panel of rows
// p0 .. n-1 and columns p0 .. p0+31 is factored in shared memory column by column (pivot, scale,
// rank-1 update of the panel's later columns), written back, and the trailing lower triangle
// takes the panel's rank-32 update in one pass over global memory, A[i][l] -= sum_c P[i][c]
// conj(P[l][c]) -- a thirty-second of the global read-modify-write passes of the column form.
// Same pivot rule and FP64 diagonal; the trailing sums are taken in a different order.
constexpr int CH_PB = 32, CH_PS = CH_PB + 1;  // panel width, panel row stride (float2)
constexpr int CH_PANEL_NMAX = 800;            // panel of n x 33 float2 + n doubles in 227 KB

__device__ void potrf_block_panel(float2* __restrict__ A, int n, int* __restrict__ status_k,
                                  int piv64, float2* P, double* dg, int& bad) {
  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  if (tid == 0) bad = 0;
  for (int i = tid; i < n; i += blockDim.x) dg[i] = (double)A[(long long)i * n + i].x;
  __syncthreads();
  for (int p0 = 0; p0 < n && !bad; p0 += CH_PB) {
    const int pw = min(CH_PB, n - p0), R = n - p0;
    // panel rows p0 .. n-1, columns p0 .. p0+pw-1 (entries above the diagonal are not used)
    for (int e = tid; e < R * pw; e += blockDim.x) {
      const int r = e / pw, c = e % pw;
      P[r * CH_PS + c] = A[(long long)(p0 + r) * n + p0 + c];
    }
    __syncthreads();
    for (int jj = 0; jj < pw; ++jj) {
      if (tid == 0) {
        const double d = piv64 ? dg[p0 + jj] : (double)P[jj * CH_PS + jj].x;
        if (!(d > 0.0) || !isfinite(d)) {
          bad = p0 + jj + 1;
        } else {
          P[jj * CH_PS + jj] = make_float2(piv64 ? (float)sqrt(d) : sqrtf((float)d), 0.f);
        }
      }
      __syncthreads();
      if (bad) break;
      const float inv = 1.f / P[jj * CH_PS + jj].x;
      for (int r = jj + 1 + tid; r < R; r += blockDim.x) {
        float2 v = P[r * CH_PS + jj];
        v.x *= inv;
        v.y *= inv;
        P[r * CH_PS + jj] = v;
        if (piv64) dg[p0 + r] -= (double)v.x * v.x + (double)v.y * v.y;
      }
      __syncthreads();
      // the panel's later columns c (rows r >= c): P[r][c] -= P[r][jj] conj(P[c][jj])
      for (int r = jj + 1 + tid; r < R; r += blockDim.x) {
        const float2 ci = P[r * CH_PS + jj];
        const int cmax = min(r, pw - 1);
        for (int c = jj + 1; c <= cmax; ++c) {
          const float2 cl = P[c * CH_PS + jj];
          float2 a = P[r * CH_PS + c];
          a.x -= ci.x * cl.x + ci.y * cl.y;
          a.y -= ci.y * cl.x - ci.x * cl.y;
          P[r * CH_PS + c] = a;
        }
      }
      __syncthreads();
    }
    if (bad) break;
    // the factored panel back to A (lower part only)
    for (int e = tid; e < R * pw; e += blockDim.x) {
      const int r = e / pw, c = e % pw;
      if (c <= r) A[(long long)(p0 + r) * n + p0 + c] = P[r * CH_PS + c];
    }
    // trailing rank-pw update, rows i and columns l beyond the panel, l <= i
    for (int i = p0 + pw + warp; i < n; i += nwarps) {
      const float2* pi = P + (i - p0) * CH_PS;
      float2* rowp = A + (long long)i * n;
      for (int l = p0 + pw + lane; l <= i; l += 32) {
        const float2* pl = P + (l - p0) * CH_PS;
        float2 sum = make_float2(0.f, 0.f);
        for (int c = 0; c < pw; ++c) {
          const float2 a = pi[c], b = pl[c];
          sum.x = fmaf(a.x, b.x, fmaf(a.y, b.y, sum.x));
          sum.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, sum.y));
        }
        float2 v = rowp[l];
        v.x -= sum.x;
        v.y -= sum.y;
        rowp[l] = v;
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

// shared memory for every matrix size up to nmax: the blocked form for n <= CH_PANEL_NMAX needs
// the panel, the column form beyond it one column; a batch may hold both kinds (217.6 KB for the
// panel of an 800-row matrix)
size_t potrf_smem(int nmax) {
  const size_t np = (size_t)std::min(nmax, CH_PANEL_NMAX);
  const size_t panel = sizeof(float2) * np * CH_PS + sizeof(double) * np;
  if (nmax <= CH_PANEL_NMAX) return panel;
  const size_t column = sizeof(float2) * (size_t)(nmax + (nmax & 1)) + sizeof(double) * (size_t)nmax;
  return std::max(panel, column);
}

__device__ inline void potrf_any(float2* A, int n, int* status_k, int piv64, float2* buf, int& bad) {
  if (n <= CH_PANEL_NMAX) {
    potrf_block_panel(A, n, status_k, piv64, buf, reinterpret_cast<double*>(buf + (size_t)n * CH_PS),
                      bad);
  } else {
    potrf_block(A, n, status_k, piv64, buf, reinterpret_cast<double*>(buf + n + (n & 1)), bad);
  }
}

__global__ void __launch_bounds__(CH_THREADS)
    k_potrf(float2* __restrict__ Lh, int n, int* __restrict__ status, int piv64) {
  extern __shared__ float2 pbuf[];  // panel (or column) cache, then the FP64 diagonal
  __shared__ int bad;
  const int k = blockIdx.x;
  potrf_any(Lh + (long long)k * n * n, n, status + k, piv64, pbuf, bad);
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
    potrf_any(it.A, it.n, it.status, piv64, col, bad);
    __syncthreads();
  }
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
  const size_t smem = potrf_smem(n);
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
