// Instantiation and launch of the yz kernels for one real type; included once
// per type by yz_f32.cu / yz_f64.cu so the two compile in parallel.
//
// Launch variants (FMMFFT_KEY_YZ_VARIANT):
//   2: team lines through shared memory, 256-thread blocks (any size; default)
//   0: lane-split register lines, 256-thread blocks (FP32, n2, n3 <= 64)
//   1: lane-split register lines, 128-thread blocks (FP32, n2, n3 <= 64)
// On the 64^3 grid variant 2 runs about twice as fast as 0 and 1: the
// register lines need ~235 registers per thread (8 warps per SM) and leave
// half the threads idle in the y pass.
// Sizes or types the lane-split kernel does not cover use variant 2; FP64
// always does (its register lines would not fit the register file).
#pragma once

#include "translate_kernels.cuh"

namespace fmm {

template <typename R, int N2, int N3, int V>
struct yz_pick {
  static constexpr bool split = V != 2 && N2 <= 64 && N3 <= 64 && sizeof(R) == 4;
  static constexpr int NT = (V == 1) ? 128 : 256;
  static constexpr int threads = split ? NT : kThreads;
  template <int FMT> static auto get() {
    if constexpr (split) return yz2_kernel<R, N2, N3, FMT, NT>;
    else return yz_kernel<R, N2, N3, FMT>;
  }
  static size_t smem(int fmt, int r2, int r3) {
    if constexpr (split) return YZ2Layout<R, N2, N3, NT>::smem_bytes(fmt, r2, r3);
    else return YZLayout<R, N2, N3>::smem_bytes(fmt, r2, r3);
  }
};

template <typename R, int N2, int N3, int FMT, int V>
cudaError_t launch_yz_v(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s) {
  static size_t configured = 0;
  using K = yz_pick<R, N2, N3, V>;
  auto kern = K::template get<FMT>();
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  kern<<<grid, K::threads, smem, s>>>(P);
  return cudaGetLastError();
}

template <typename R, int N2, int N3, int FMT>
cudaError_t launch_yz_inst(const YZParams& P, dim3 grid, size_t smem, cudaStream_t s) {
  if constexpr (!yz_pick<R, N2, N3, 0>::split) {
    return launch_yz_v<R, N2, N3, FMT, 2>(P, grid, smem, s);
  } else {
    if (P.variant == 1) return launch_yz_v<R, N2, N3, FMT, 1>(P, grid, smem, s);
    if (P.variant == 2) return launch_yz_v<R, N2, N3, FMT, 2>(P, grid, smem, s);
    return launch_yz_v<R, N2, N3, FMT, 0>(P, grid, smem, s);
  }
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

template <typename R, int N2, int N3>
size_t yz_smem_inst(int fmt, int r2, int r3, int variant) {
  if (!yz_pick<R, N2, N3, 0>::split || variant == 2) return yz_pick<R, N2, N3, 2>::smem(fmt, r2, r3);
  if (variant == 1) return yz_pick<R, N2, N3, 1>::smem(fmt, r2, r3);
  return yz_pick<R, N2, N3, 0>::smem(fmt, r2, r3);
}

template <typename R, int N2>
size_t yz_smem_n3(int n3, int fmt, int r2, int r3, int variant) {
  switch (n3) {
    case 4: return yz_smem_inst<R, N2, 4>(fmt, r2, r3, variant);
    case 8: return yz_smem_inst<R, N2, 8>(fmt, r2, r3, variant);
    case 16: return yz_smem_inst<R, N2, 16>(fmt, r2, r3, variant);
    case 32: return yz_smem_inst<R, N2, 32>(fmt, r2, r3, variant);
    case 64: return yz_smem_inst<R, N2, 64>(fmt, r2, r3, variant);
    case 128: return yz_smem_inst<R, N2, 128>(fmt, r2, r3, variant);
    default: return 0;
  }
}

template <typename R>
size_t yz_smem_any(int n2, int n3, int fmt, int r2, int r3, int variant) {
  switch (n2) {
    case 4: return yz_smem_n3<R, 4>(n3, fmt, r2, r3, variant);
    case 8: return yz_smem_n3<R, 8>(n3, fmt, r2, r3, variant);
    case 16: return yz_smem_n3<R, 16>(n3, fmt, r2, r3, variant);
    case 32: return yz_smem_n3<R, 32>(n3, fmt, r2, r3, variant);
    case 64: return yz_smem_n3<R, 64>(n3, fmt, r2, r3, variant);
    case 128: return yz_smem_n3<R, 128>(n3, fmt, r2, r3, variant);
    default: return 0;
  }
}

}  // namespace fmm
