// yz-pass kernels, FP32 fields (complex64).
#include "yz_dispatch.cuh"

namespace fmm {
cudaError_t launch_yz_f32(const YZParams& P, int n2, int n3, int fmt, dim3 grid, size_t smem,
                          cudaStream_t s) {
  return launch_yz_any<float>(P, n2, n3, fmt, grid, smem, s);
}
size_t yz_smem_f32(int n2, int n3, int fmt, int r2, int r3, int variant) {
  return yz_smem_any<float>(n2, n3, fmt, r2, r3, variant);
}
}  // namespace fmm
