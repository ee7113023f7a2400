// Internal plan state shared by the host set-up code and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <complex>
#include <vector>

#include "../../include/fmmfft.h"

namespace fmm {

using cdouble = std::complex<double>;

// Per-direction Tucker-3D descriptor (device and host copies).  Offsets count
// complex elements in the packed factor buffer / the restore scratch buffer.
struct Tucker3DDesc {
  int r1, r2, r3, pad;
  int64_t off_core;   // C_p, r1 x r2 x r3, c fastest
  int64_t off_u1;     // U1_p, n1 x r1
  int64_t off_u2;     // U2_p, n2 x r2
  int64_t off_u3;     // U3_p, n3 x r3
  int64_t off_h;      // H_p = C_p x_1 U1_p, n1 x r2 x r3, in the restore scratch
};

// Arguments of one translation, prepared by the host for the launchers.
struct TranslateArgs {
  int K[3];           // Kx, Ky, Kz
  int n[3];           // n1, n2, n3
  int n_dir;
  int nrhs;
  int precision;      // FMMFFT_PREC_*
  int format, decomp;
  const void* s_in;
  void* s_out;
  void* inter;        // x-transformed fields, [F][n1][Kz][Ky]
  const void* tw[3];  // twiddle tables W_{n_i}^m, m < n_i
  // format NONE: T~_p / (n1 n2 n3), layout [p][x][z][y]
  const void* op_plain;
  // Tucker-3D
  const Tucker3DDesc* t3_desc;   // device, n_dir entries
  const void* t3_pack;           // device, packed cores and factors
  void* t3_h;                    // device, restore scratch (H_p)
  int t3_rmax[3];                // largest r1, r2, r3
  int* status;                   // device status word
  cudaEvent_t* events;           // FMMFFT_NUM_STAGES + 1 events, or null
  int yz_variant;                // FMMFFT_KEY_YZ_VARIANT
  cudaStream_t stream;
};

// Kernel launchers (translate_kernels.cu).  Return a cudaError_t.
cudaError_t launch_translate(const TranslateArgs& a);
// Largest shared-memory request of the yz kernel for the given args (bytes);
// 0 if the sizes are not supported by the compiled kernels.
size_t yz_smem_bytes(const TranslateArgs& a);
bool translate_supported(const TranslateArgs& a);

// Translation of a compressed plan with a caller-provided intermediate buffer
// (fmmfft_api.cpp), used by the allocation-free entry point.
// translate_scratch_bytes validates the plan and nrhs and returns the bytes of
// intermediate one call needs; translate_into validates the field buffers and
// launches the translation with `scratch` (scratch_bytes long) as intermediate.
int translate_scratch_bytes(fmmfft_plan p, int nrhs, size_t* bytes);
int translate_into(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* stream,
                   void* scratch, size_t scratch_bytes);

}  // namespace fmm
