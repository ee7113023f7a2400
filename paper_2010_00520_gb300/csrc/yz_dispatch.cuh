// Instantiation and launch of the yz kernel for one real type and one operator
// format; included once per (type, format) by the yz_*.cu units so that they
// compile in parallel.
#pragma once

#include "translate_kernels.cuh"

namespace fmm {

// Single translation (inst = null, the given grid) or batch mode (inst, ninst
// instances of this shape class, `total` items, one block per item).
template <typename R, int N2, int N3, int FMT, int TC>
cudaError_t launch_yz_tc(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s, const BatchYZ* inst = nullptr,
                         int ninst = 0, long long total = 0) {
  static std::atomic<int> optin[kMaxDevices];
  auto kern = yz_kernel<R, N2, N3, FMT, TC>;
  cudaError_t e = smem_optin((const void*)kern, optin);
  if (e != cudaSuccess) return e;
  // batch mode: one block per item (the kernel's item loop runs once)
  if (inst) {
    if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
    grid = dim3((unsigned)total);
  }
  kern<<<grid, kThreads, smem, s>>>(P, inst, ninst, total);
  return cudaGetLastError();
}

template <typename R, int N2, int N3, int FMT>
cudaError_t launch_yz_inst(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s, const BatchYZ* inst,
                           int ninst, long long total) {
  if constexpr (TcRestore<R, N2, N3, FMT>::available) {
    if (P.tc == 1) return launch_yz_tc<R, N2, N3, FMT, 1>(P, grid, smem, s, inst, ninst, total);
    if (P.tc == 2) return launch_yz_tc<R, N2, N3, FMT, 2>(P, grid, smem, s, inst, ninst, total);
  }
  return launch_yz_tc<R, N2, N3, FMT, 0>(P, grid, smem, s, inst, ninst, total);
}

template <typename R, int FMT, int N2>
cudaError_t launch_yz_n3(const YZParams& P, int n3, dim3 grid, size_t smem, cudaStream_t s, const BatchYZ* inst,
                         int ninst, long long total) {
  switch (n3) {
    case 4: return launch_yz_inst<R, N2, 4, FMT>(P, grid, smem, s, inst, ninst, total);
    case 8: return launch_yz_inst<R, N2, 8, FMT>(P, grid, smem, s, inst, ninst, total);
    case 16: return launch_yz_inst<R, N2, 16, FMT>(P, grid, smem, s, inst, ninst, total);
    case 32: return launch_yz_inst<R, N2, 32, FMT>(P, grid, smem, s, inst, ninst, total);
    case 64: return launch_yz_inst<R, N2, 64, FMT>(P, grid, smem, s, inst, ninst, total);
    case 128: return launch_yz_inst<R, N2, 128, FMT>(P, grid, smem, s, inst, ninst, total);
    default: return cudaErrorInvalidValue;
  }
}

// P: the parameters of a single translation, or in batch mode (inst != null)
// those of any instance of the class (its tc field picks the kernel)
template <typename R, int FMT>
cudaError_t launch_yz_fmt(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, cudaStream_t s,
                          const BatchYZ* inst = nullptr, int ninst = 0, long long total = 0) {
  switch (n2) {
    case 4: return launch_yz_n3<R, FMT, 4>(P, n3, grid, smem, s, inst, ninst, total);
    case 8: return launch_yz_n3<R, FMT, 8>(P, n3, grid, smem, s, inst, ninst, total);
    case 16: return launch_yz_n3<R, FMT, 16>(P, n3, grid, smem, s, inst, ninst, total);
    case 32: return launch_yz_n3<R, FMT, 32>(P, n3, grid, smem, s, inst, ninst, total);
    case 64: return launch_yz_n3<R, FMT, 64>(P, n3, grid, smem, s, inst, ninst, total);
    case 128: return launch_yz_n3<R, FMT, 128>(P, n3, grid, smem, s, inst, ninst, total);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R, int N2, int N3, int FMT, int TC>
cudaError_t launch_yzl_tc(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s) {
  static std::atomic<int> optin[kMaxDevices];
  auto kern = yzl_kernel<R, N2, N3, FMT, TC>;
  cudaError_t e = smem_optin((const void*)kern, optin);
  if (e != cudaSuccess) return e;
  kern<<<grid, kThreads, smem, s>>>(P);
  return cudaGetLastError();
}

template <typename R, int N2, int N3, int FMT>
cudaError_t launch_yzl_inst(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s) {
  if constexpr (TcRestore<R, N2, N3, FMT>::available) {
    if (P.tc == 1) return launch_yzl_tc<R, N2, N3, FMT, 1>(P, grid, smem, s);
    if (P.tc == 2) return launch_yzl_tc<R, N2, N3, FMT, 2>(P, grid, smem, s);
  }
  return launch_yzl_tc<R, N2, N3, FMT, 0>(P, grid, smem, s);
}

// Large-plane shapes (slab and plane do not fit shared memory together).
template <typename R, int FMT>
cudaError_t launch_yzl_fmt(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, cudaStream_t s) {
  if (n2 == 128 && n3 == 128) return launch_yzl_inst<R, 128, 128, FMT>(P, grid, smem, s);
  if (n2 == 256 && n3 == 64) return launch_yzl_inst<R, 256, 64, FMT>(P, grid, smem, s);
  if (n2 == 256 && n3 == 128) return launch_yzl_inst<R, 256, 128, FMT>(P, grid, smem, s);
  return cudaErrorInvalidValue;
}

}  // namespace fmm

// One translation unit per (type, format).
#define FMM_YZ_UNIT(R, TAG, FMT)                                                             \
  namespace fmm {                                                                            \
  cudaError_t launch_yz_##TAG##_##FMT(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, \
                                      cudaStream_t s) {                                      \
    return launch_yz_fmt<R, FMT>(P, n2, n3, grid, smem, s);                                  \
  }                                                                                          \
  cudaError_t launch_yzl_##TAG##_##FMT(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, \
                                       cudaStream_t s) {                                     \
    return launch_yzl_fmt<R, FMT>(P, n2, n3, grid, smem, s);                                 \
  }                                                                                          \
  cudaError_t launch_yz_batch_##TAG##_##FMT(const YZParams& P, int n2, int n3, size_t smem,   \
                                            cudaStream_t s, const BatchYZ* inst, int ninst,  \
                                            long long total) {                               \
    return launch_yz_fmt<R, FMT>(P, n2, n3, dim3(1), smem, s, inst, ninst, total);           \
  }                                                                                          \
  }
