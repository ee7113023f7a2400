// Instantiation and launch of the yz kernels for one real type; included once
// per type by yz_f32.cu / yz_f64.cu so the two compile in parallel.
#pragma once

#include "translate_kernels.cuh"

namespace fmm {

template <typename R, int N2, int N3, int FMT>
cudaError_t launch_yz_inst(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s) {
  static size_t configured = 0;
  auto kern = yz_kernel<R, N2, N3, FMT>;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  kern<<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

template <typename R, int N2>
cudaError_t launch_yz_n3(const YZParams& P, int n3, int fmt, dim3 grid, size_t smem, cudaStream_t s) {
#define FMM_YZ_CASE(N3)                                                         \
  case N3:                                                                      \
    return fmt == 0 ? launch_yz_inst<R, N2, N3, 0>(P, grid, smem, s)            \
                    : launch_yz_inst<R, N2, N3, 1>(P, grid, smem, s);
  switch (n3) {
    FMM_YZ_CASE(4) FMM_YZ_CASE(8) FMM_YZ_CASE(16) FMM_YZ_CASE(32) FMM_YZ_CASE(64) FMM_YZ_CASE(128)
    default: return cudaErrorInvalidValue;
  }
#undef FMM_YZ_CASE
}

template <typename R>
cudaError_t launch_yz_any(const YZParams& P, int n2, int n3, int fmt, dim3 grid, size_t smem,
                          cudaStream_t s) {
  switch (n2) {
    case 4: return launch_yz_n3<R, 4>(P, n3, fmt, grid, smem, s);
    case 8: return launch_yz_n3<R, 8>(P, n3, fmt, grid, smem, s);
    case 16: return launch_yz_n3<R, 16>(P, n3, fmt, grid, smem, s);
    case 32: return launch_yz_n3<R, 32>(P, n3, fmt, grid, smem, s);
    case 64: return launch_yz_n3<R, 64>(P, n3, fmt, grid, smem, s);
    case 128: return launch_yz_n3<R, 128>(P, n3, fmt, grid, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int N2>
size_t yz_smem_n3(int n3, int fmt, int r2, int r3) {
  switch (n3) {
    case 4: return YZLayout<R, N2, 4>::smem_bytes(fmt, r2, r3);
    case 8: return YZLayout<R, N2, 8>::smem_bytes(fmt, r2, r3);
    case 16: return YZLayout<R, N2, 16>::smem_bytes(fmt, r2, r3);
    case 32: return YZLayout<R, N2, 32>::smem_bytes(fmt, r2, r3);
    case 64: return YZLayout<R, N2, 64>::smem_bytes(fmt, r2, r3);
    case 128: return YZLayout<R, N2, 128>::smem_bytes(fmt, r2, r3);
    default: return 0;
  }
}

template <typename R>
size_t yz_smem_any(int n2, int n3, int fmt, int r2, int r3) {
  switch (n2) {
    case 4: return yz_smem_n3<R, 4>(n3, fmt, r2, r3);
    case 8: return yz_smem_n3<R, 8>(n3, fmt, r2, r3);
    case 16: return yz_smem_n3<R, 16>(n3, fmt, r2, r3);
    case 32: return yz_smem_n3<R, 32>(n3, fmt, r2, r3);
    case 64: return yz_smem_n3<R, 64>(n3, fmt, r2, r3);
    case 128: return yz_smem_n3<R, 128>(n3, fmt, r2, r3);
    default: return 0;
  }
}

}  // namespace fmm
