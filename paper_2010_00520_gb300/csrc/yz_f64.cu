// yz-pass kernels, FP64 fields (complex128).
#include "yz_dispatch.cuh"

namespace fmm {
cudaError_t launch_yz_f64(const YZParams& P, int n2, int n3, int fmt, dim3 grid, size_t smem,
                          cudaStream_t s) {
  return launch_yz_any<double>(P, n2, n3, fmt, grid, smem, s);
}
size_t yz_smem_f64(int n2, int n3, int fmt, int r2, int r3, int variant) {
  return yz_smem_any<double>(n2, n3, fmt, r2, r3, variant);
}
}  // namespace fmm
