// Allocation-free entry point for the per-frequency Gram (egh_gram_noalloc, include/egh.h).
//
// Some callers cannot call cudaMalloc: a process whose device memory is already fully reserved
// by another allocator (a framework's caching pool or an arena sized at start-up), or a service
// loop that forbids device allocation (and the implicit synchronisation of cudaMalloc/cudaFree)
// once it is running.  For them this entry point runs the same Gram kernels as egh_hessian but
// takes the split-sum workspace from a fixed array in device memory that the library defines
// at file scope.  CUDA loads this file's device code lazily (on first use, by default), so the
// array's 32 MiB are reserved on a device by the first call there and held until the process
// exits; callers make that first call at start-up, before their own allocator takes the memory.
//
// In host code `g_gram_scratch` names a host-side stand-in, not device memory: its device
// address is obtained with cudaGetSymbolAddress once per device (on the first call made while
// that device is current) and passed to the kernels.
#include <algorithm>
#include <cstdint>
#include <mutex>
#include <string>

#include "egh.h"
#include "egh_internal.cuh"

namespace {

// 8 Mi floats = 32 MiB of split-sum workspace per device.
constexpr size_t kScratchFloats = size_t(8) << 20;
__device__ __align__(256) float g_gram_scratch[kScratchFloats];

constexpr int kMaxDevices = 64;
float* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_on_current_device(float** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_gram_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = static_cast<float*>(p);
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

bool is_device_pointer(const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

egh_status fail(egh_status s, const std::string& msg) {
  egh::set_context_free_error(msg);
  return s;
}

}  // namespace

extern "C" egh_status egh_gram_noalloc(const float* gh, int32_t nrec, int32_t nfreq, int64_t npts,
                                       void* H, void* stream) {
  if (!gh || !H) return fail(EGH_EINVAL, "egh_gram_noalloc: NULL buffer");
  if (nrec < 1 || nfreq < 1) return fail(EGH_EINVAL, "egh_gram_noalloc: nrec and nfreq must be >= 1");
  if (npts < 16 || npts % 16 != 0)
    return fail(EGH_EINVAL, "egh_gram_noalloc: npts must be a positive multiple of 16");
  if ((reinterpret_cast<uintptr_t>(gh) & 15) || (reinterpret_cast<uintptr_t>(H) & 7))
    return fail(EGH_EINVAL, "egh_gram_noalloc: gh must be 16-byte and H 8-byte aligned");
  if (!is_device_pointer(gh) || !is_device_pointer(H))
    return fail(EGH_EINVAL, "egh_gram_noalloc: gh and H must be device memory");
  const size_t one_split = egh::gram_workspace_floats(nrec, nfreq, 1);
  if (one_split > kScratchFloats) {
    return fail(EGH_EINVAL,
                "egh_gram_noalloc: nrec = " + std::to_string(nrec) + ", nfreq = " +
                    std::to_string(nfreq) + " needs " + std::to_string(one_split) +
                    " floats of workspace; the fixed scratch holds " +
                    std::to_string(kScratchFloats) + " (nfreq x tile pairs <= 2048, tile = 32 "
                    "receivers)");
  }
  float* scratch = nullptr;
  cudaError_t e = scratch_on_current_device(&scratch);
  if (e != cudaSuccess)
    return fail(EGH_ECUDA, std::string("egh_gram_noalloc: cudaGetSymbolAddress: ") +
                               cudaGetErrorString(e));
  // as many splits of the grid sum as fit the scratch, up to the default heuristic
  const int ntile = egh::gram_tiles(nrec);
  const long long pairs_nf = (long long)ntile * (ntile + 1) / 2 * nfreq;
  long long want = (3LL * 456 + pairs_nf - 1) / pairs_nf;
  want = std::max(1LL, std::min(want, (long long)(npts / 2048)));
  const long long fit = (long long)(kScratchFloats / one_split);
  const int splits = (int)std::max(1LL, std::min(want, fit));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  e = egh::launch_gram_partial(gh, nrec, nfreq, npts, splits, scratch, st);
  if (e == cudaSuccess)
    e = egh::launch_gram_finish(scratch, nrec, nfreq, splits, static_cast<float2*>(H), st);
  if (e != cudaSuccess)
    return fail(EGH_ECUDA, std::string("egh_gram_noalloc: launch: ") + cudaGetErrorString(e));
  return EGH_OK;
}
