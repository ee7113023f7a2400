// fmmfft_translate_noalloc: the translation with its intermediate buffer in a
// fixed file-scope device array instead of memory the plan allocates.
//
// It serves callers that cannot call cudaMalloc while translating (a solver
// inside a framework whose pool owns the device memory, or a time-critical
// loop where an allocation would synchronise the device).  The array below is
// part of this library's device image: each GPU that loads the library holds
// its FMMFFT_NOALLOC_SCRATCH_BYTES until the process exits, and every call
// shares it, so calls whose kernels overlap on the GPU race on it.  Nothing
// in it needs clearing: the x pass of a call writes every element the later
// passes read.
#include <mutex>

#include "../../include/fmmfft.h"
#include "plan_internal.h"

static __device__ __align__(256) unsigned char g_translate_scratch[FMMFFT_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_scratch_mutex;
void* g_scratch_addr[fmm::kMaxDevices] = {};

// Device address of g_translate_scratch on the current device.  In host code
// the array's name stands for a host-side shadow, not device memory, so the
// address comes from the runtime once per device and is cached.  The cache is
// tied to the context the first call saw: a cudaDeviceReset invalidates it
// (the header tells callers not to use this entry point after a reset).
int scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  if (dev < 0 || dev >= fmm::kMaxDevices) return FMMFFT_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_translate_scratch);
    if (e != cudaSuccess || !ptr) {
      cudaGetLastError();
      return FMMFFT_ERR_CUDA;
    }
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return FMMFFT_OK;
}

}  // namespace

extern "C" int fmmfft_translate_noalloc(fmmfft_plan plan, const void* S_in, void* S_out, int nrhs,
                                        void* stream) {
  size_t need = 0;
  int st = fmm::translate_scratch_bytes(plan, nrhs, &need);
  if (st != FMMFFT_OK) return st;
  if (need > FMMFFT_NOALLOC_SCRATCH_BYTES) return FMMFFT_ERR_TOO_LARGE;
  void* scratch = nullptr;
  if ((st = scratch_address(&scratch)) != FMMFFT_OK) return st;
  return fmm::translate_into(plan, S_in, S_out, nrhs, stream, scratch, FMMFFT_NOALLOC_SCRATCH_BYTES);
}
