// Deblurring of residual gathers against the factored Hessians (eq. Qsystem solved per frequency,
// Section "Frequency domain inversion"):
//   D[k][r][s] = sum_t resid[s][r][t] exp(-i w_k t dt)           (k_trace_dft)
//   X_k = L_k^{-H} L_k^{-1} D_k                                   (k_trsm, all sources as RHS)
//   mixed precision: X_k += L_k^{-H} L_k^{-1} (D_k - Q_k X_k)      (k_resid64 in FP64, k_trsm)
//   mult[s][r][t] = sum_k w_k Re(X_k[r][s] exp(+i w_k t dt))      (k_synth)
// Traces are indexed q = s * nrec + r (the [ns][nrec][nt] gather layout); the spectra of one call
// occupy columns s0 .. s0 + ns - 1 of a [nf][nrec][ld] array, so that several gathers (of
// different lengths) can share one solve.
#include <algorithm>

#include "egh_internal.cuh"

namespace egh {

constexpr int NFMAX = 64;

// ---------------------------------------------------------------------------------------------
// Forward transform: 64 traces per block, the time axis staged 64 samples at a time with the
// twiddles of the stage in shared memory.  Thread (m, g) accumulates trace m at frequencies
// k = g, g+4, ...; each stage's partial sum is added into the running total (two-level sum).
// ---------------------------------------------------------------------------------------------
constexpr int TD_TR = 64, TD_T = 64;

__global__ void __launch_bounds__(256)
    k_trace_dft(const float* __restrict__ resid, int ntr, int nt_d, const float2* __restrict__ tw,
                int nf, int nrec, int ld, int s0, float2* __restrict__ Dh) {
  __shared__ float R[TD_TR][TD_T + 1];
  extern __shared__ float2 stw[];  // [TD_T][nf]
  const int tid = threadIdx.x, m = tid & 63, g = tid >> 6;
  const int q0 = blockIdx.x * TD_TR;
  float2 tot[NFMAX / 4];
#pragma unroll
  for (int j = 0; j < NFMAX / 4; ++j) tot[j] = make_float2(0.f, 0.f);
  for (int t0 = 0; t0 < nt_d; t0 += TD_T) {
#pragma unroll 4
    for (int i = 0; i < (TD_TR * TD_T) / 256; ++i) {
      const int e = tid + 256 * i;
      const int r = e >> 6, c = e & 63;
      const int q = q0 + r, t = t0 + c;
      R[r][c] = (q < ntr && t < nt_d) ? resid[(long long)q * nt_d + t] : 0.f;
    }
    for (int e = tid; e < TD_T * nf; e += 256) {
      const int t = t0 + e / nf;
      stw[e] = t < nt_d ? tw[(long long)t0 * nf + e] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[NFMAX / 4];
#pragma unroll
    for (int j = 0; j < NFMAX / 4; ++j) acc[j] = make_float2(0.f, 0.f);
    for (int tt = 0; tt < TD_T; ++tt) {
      const float x = R[m][tt];
#pragma unroll
      for (int j = 0; j < NFMAX / 4; ++j) {
        const int k = g + 4 * j;
        if (k < nf) {
          const float2 w = stw[tt * nf + k];
          acc[j].x = fmaf(x, w.x, acc[j].x);
          acc[j].y = fmaf(x, w.y, acc[j].y);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < NFMAX / 4; ++j) {
      tot[j].x += acc[j].x;
      tot[j].y += acc[j].y;
    }
    __syncthreads();
  }
  const int q = q0 + m;
  if (q < ntr) {
    const int s = q / nrec, r = q % nrec;
#pragma unroll
    for (int j = 0; j < NFMAX / 4; ++j) {
      const int k = g + 4 * j;
      if (k < nf) Dh[((long long)k * nrec + r) * ld + s0 + s] = tot[j];
    }
  }
}

cudaError_t launch_trace_dft(const float* resid, int ntr, int nt_d, const float2* tw, int nf,
                             int nrec, int ld, int s0, float2* Dh, cudaStream_t st) {
  if (nf > NFMAX) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float2) * TD_T * nf;
  if (smem + sizeof(float) * TD_TR * (TD_T + 1) > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_trace_dft, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_trace_dft<<<(ntr + TD_TR - 1) / TD_TR, 256, smem, st>>>(resid, ntr, nt_d, tw, nf, nrec, ld, s0,
                                                          Dh);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Triangular solves L y = d, L^H x = y for 32 right-hand sides (sources) per block, one block per
// (frequency, column group).  The RHS block lives in shared memory; for each row the dot product
// over earlier rows is split across the eight warps and reduced through shared memory.
// ---------------------------------------------------------------------------------------------
constexpr int TS_W = 8;

__device__ inline float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ inline float2 cmulc(float2 a, float2 b) {  // conj(a) * b
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}

__global__ void __launch_bounds__(32 * TS_W)
    k_trsm(const float2* __restrict__ Lh, int n, float2* __restrict__ Dh, int ns) {
  extern __shared__ float2 Y[];  // [n][32]
  __shared__ float2 red[TS_W][32];
  const int k = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool valid = col < ns;
  const float2* L = Lh + (long long)k * n * n;
  float2* B = Dh + (long long)k * n * ns;
  for (int i = warp; i < n; i += TS_W)
    Y[i * 32 + lane] = valid ? B[(long long)i * ns + col] : make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = 0; i < n; ++i) {
    float2 s = make_float2(0.f, 0.f);
    for (int j = warp; j < i; j += TS_W) {
      const float2 p = cmul(L[(long long)i * n + j], Y[j * 32 + lane]);
      s.x += p.x;
      s.y += p.y;
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      float2 t = Y[i * 32 + lane];
#pragma unroll
      for (int w = 0; w < TS_W; ++w) {
        t.x -= red[w][lane].x;
        t.y -= red[w][lane].y;
      }
      const float d = 1.f / L[(long long)i * n + i].x;
      Y[i * 32 + lane] = make_float2(t.x * d, t.y * d);
    }
    __syncthreads();
  }
  for (int i = n - 1; i >= 0; --i) {
    float2 s = make_float2(0.f, 0.f);
    for (int j = i + 1 + warp; j < n; j += TS_W) {
      const float2 p = cmulc(L[(long long)j * n + i], Y[j * 32 + lane]);
      s.x += p.x;
      s.y += p.y;
    }
    red[warp][lane] = s;
    __syncthreads();
    if (warp == 0) {
      float2 t = Y[i * 32 + lane];
#pragma unroll
      for (int w = 0; w < TS_W; ++w) {
        t.x -= red[w][lane].x;
        t.y -= red[w][lane].y;
      }
      const float d = 1.f / L[(long long)i * n + i].x;
      Y[i * 32 + lane] = make_float2(t.x * d, t.y * d);
    }
    __syncthreads();
  }
  if (valid)
    for (int i = warp; i < n; i += TS_W) B[(long long)i * ns + col] = Y[i * 32 + lane];
}

cudaError_t launch_trsm(const float2* Lh, int n, int nf, float2* Dh, int ns, cudaStream_t st) {
  const size_t smem = sizeof(float2) * 32 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_trsm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((ns + 31) / 32, nf);
  count_launches(1);
  k_trsm<<<grid, 32 * TS_W, smem, st>>>(Lh, n, Dh, ns);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------------
// Synthesis: 64 traces x 128 samples per block.  The weighted solutions of the block's traces and
// the twiddles of its time range sit in shared memory; thread (t, half) produces sample t of 32
// traces.  Re(X e^{+i theta}) = Re X cos(theta) + Im X (-sin(theta)) with tw = e^{-i theta}.
// ---------------------------------------------------------------------------------------------
constexpr int SY_TR = 64, SY_T = 128;

__global__ void __launch_bounds__(256)
    k_synth(const float2* __restrict__ Dh, int nrec, int ld, int s0, int nf,
            const float* __restrict__ w, const float2* __restrict__ tw, int nt_d,
            float* __restrict__ mult, int ntr) {
  extern __shared__ float2 sm[];
  float2* X = sm;                 // [SY_TR][nf]
  float2* T = sm + SY_TR * nf;    // [nf][SY_T]
  const int tid = threadIdx.x;
  const int q0 = blockIdx.y * SY_TR, t0 = blockIdx.x * SY_T;
  for (int e = tid; e < SY_TR * nf; e += 256) {
    const int rr = e / nf, k = e % nf, q = q0 + rr;
    float2 v = make_float2(0.f, 0.f);
    if (q < ntr) {
      v = Dh[((long long)k * nrec + q % nrec) * ld + s0 + q / nrec];
      v.x *= w[k];
      v.y *= w[k];
    }
    X[e] = v;
  }
  for (int e = tid; e < nf * SY_T; e += 256) {
    const int k = e / SY_T, tt = e % SY_T, t = t0 + tt;
    T[e] = t < nt_d ? tw[(long long)t * nf + k] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  const int tl = tid & (SY_T - 1), half = tid >> 7;
  float acc[32];
#pragma unroll
  for (int m = 0; m < 32; ++m) acc[m] = 0.f;
  for (int k = 0; k < nf; ++k) {
    const float2 c = T[k * SY_T + tl];
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      const float2 x = X[(half * 32 + m) * nf + k];
      acc[m] = fmaf(x.x, c.x, fmaf(x.y, c.y, acc[m]));
    }
  }
  const int t = t0 + tl;
  if (t < nt_d) {
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      const int q = q0 + half * 32 + m;
      if (q < ntr) mult[(long long)q * nt_d + t] = acc[m];
    }
  }
}

// ---------------------------------------------------------------------------------------------
// Refinement residual in FP64: R_k = D_k - Q_k X_k, products of the FP32 operands (exact in FP64)
// accumulated in double and rounded once (mixed-precision iterative refinement of the solves).
// One block per (frequency, 32 sources, group of rows); X_k's columns sit in shared memory;
// warp w takes rows w, w + 8, ... of its group; lane = source.
// ---------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * TS_W)
    k_resid64(const float2* __restrict__ Qh, int n, const float2* __restrict__ Xh,
              const float2* __restrict__ Dh, int ns, float2* __restrict__ Rh) {
  extern __shared__ float2 Xs[];  // [n][32]
  const int k = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int col = blockIdx.x * 32 + lane;
  const bool valid = col < ns;
  const float2* Q = Qh + (long long)k * n * n;
  const long long off = (long long)k * n * ns;
  for (int i = warp; i < n; i += TS_W)
    Xs[i * 32 + lane] = valid ? Xh[off + (long long)i * ns + col] : make_float2(0.f, 0.f);
  __syncthreads();
  const int rows = (n + gridDim.z - 1) / gridDim.z;
  const int i0 = blockIdx.z * rows, i1 = min(n, i0 + rows);
  for (int i = i0 + warp; i < i1; i += TS_W) {
    double re = 0.0, im = 0.0;
    const float2* q = Q + (long long)i * n;
    for (int j = 0; j < n; ++j) {
      const float2 a = q[j], x = Xs[j * 32 + lane];
      re = fma((double)a.x, (double)x.x, fma(-(double)a.y, (double)x.y, re));
      im = fma((double)a.x, (double)x.y, fma((double)a.y, (double)x.x, im));
    }
    if (valid) {
      const float2 d = Dh[off + (long long)i * ns + col];
      Rh[off + (long long)i * ns + col] = make_float2((float)((double)d.x - re), (float)((double)d.y - im));
    }
  }
}

cudaError_t launch_resid64(const float2* Qh, int n, int nf, const float2* Xh, const float2* Dh,
                           int ns, float2* Rh, cudaStream_t st) {
  const size_t smem = sizeof(float2) * 32 * (size_t)n;
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_resid64, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  // enough blocks for every SM: split the rows of each (frequency, source group)
  const int blocks = ((ns + 31) / 32) * nf;
  const int groups = std::max(1, std::min((n + TS_W - 1) / TS_W, (4 * 152 + blocks - 1) / blocks));
  k_resid64<<<dim3((ns + 31) / 32, nf, groups), 32 * TS_W, smem, st>>>(Qh, n, Xh, Dh, ns, Rh);
  return cudaGetLastError();
}

// X += R (complex, all frequencies and sources)
__global__ void k_add_correction(float2* __restrict__ X, const float2* __restrict__ R, long long m) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < m;
       i += (long long)gridDim.x * blockDim.x) {
    const float2 r = R[i];
    float2 x = X[i];
    x.x += r.x;
    x.y += r.y;
    X[i] = x;
  }
}

cudaError_t launch_add_correction(float2* X, const float2* R, long long m, cudaStream_t st) {
  long long blocks = (m + 255) / 256;
  if (blocks > 4096) blocks = 4096;
  count_launches(1);
  k_add_correction<<<(int)blocks, 256, 0, st>>>(X, R, m);
  return cudaGetLastError();
}

cudaError_t launch_synth(const float2* Dh, int nrec, int ns, int ld, int s0, int nf, const float* w,
                         const float2* tw, int nt_d, float* mult, cudaStream_t st) {
  if (nf > NFMAX) return cudaErrorInvalidValue;
  const int ntr = nrec * ns;
  const size_t smem = sizeof(float2) * (size_t)nf * (SY_TR + SY_T);
  if (smem > 48 * 1024) {
    cudaError_t e =
        cudaFuncSetAttribute(k_synth, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((nt_d + SY_T - 1) / SY_T, (ntr + SY_TR - 1) / SY_TR);
  count_launches(1);
  k_synth<<<grid, 256, smem, st>>>(Dh, nrec, ld, s0, nf, w, tw, nt_d, mult, ntr);
  return cudaGetLastError();
}

}  // namespace egh
