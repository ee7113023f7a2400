// Internal plan state shared by the host set-up code and the kernel launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <complex>
#include <vector>

#include "../../include/fmmfft.h"

namespace fmm {

using cdouble = std::complex<double>;

// Devices a process may drive (per-device launch state below).
constexpr int kMaxDevices = 64;

// Let `func` take up to the device's opt-in maximum of dynamic shared memory
// (less its static shared memory), once per device: `done` is the caller's
// per-kernel array of kMaxDevices flags (static storage, zero-initialised).
// The attribute is a per-device upper bound, so one setting serves every
// later launch size; setting it twice (two threads) is harmless.
inline cudaError_t smem_optin(const void* func, std::atomic<int>* done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const bool cache = dev >= 0 && dev < kMaxDevices;
  if (cache && done[dev].load(std::memory_order_acquire)) return cudaSuccess;
  int optin = 0;
  if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
  cudaFuncAttributes fa;
  if ((e = cudaFuncGetAttributes(&fa, func)) != cudaSuccess) return e;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e == cudaSuccess && cache) done[dev].store(1, std::memory_order_release);
  return e;
}

// Per-direction restore descriptor of the yz kernel (device pointers).
//   Tucker-like (yz format 1): h = H_p, row x at h + x * hx (ra x rb, [b][c]);
//                              u2 = U2 (n2 x ra); u3 = U3 (n3 x rb)
//   TT-like (yz format 2):     h = T1 of the direction, row x at h + x * hx
//                              (n2 x rb, [y][b]); u3 = R_p (n3 x rb); ra = 0
struct SlabDesc {
  const void* h;
  const void* u2;
  const void* u3;
  long long hx;
  int ra, rb;
};

// One product of the restore pre-pass: C = A B, complex, row-major and
// contiguous (A: M x K, B: K x N, C: M x N).
struct GemmDesc {
  const void* A;
  const void* B;
  void* C;
  int M, N, K, pad;
};

// One launch of the pre-pass: `batch` products described at `desc` (device).
struct GemmStage {
  const GemmDesc* desc;
  int batch;
  int max_m, max_n;
};

constexpr int kMaxGemmStages = 4;

struct XDisArgs;

// Arguments of one translation, prepared by the host for the launchers.
struct TranslateArgs {
  int K[3];           // Kx, Ky, Kz
  int n[3];           // n1, n2, n3
  int n_dir;
  int nrhs;
  int precision;      // FMMFFT_PREC_*
  int yz_fmt;         // 0 plain operator, 1 Tucker-like restore, 2 TT-like restore
  const void* s_in;
  void* s_out;
  void* inter;        // x-transformed fields, [F][n1][Kz][Ky]
  const void* tw[3];  // twiddle tables W_{n_i}^m, m < n_i
  // format NONE: T~_p / (n1 n2 n3), layout [p][x][z][y]
  const void* op_plain;
  // compressed formats
  const SlabDesc* slab;              // device, n_dir entries
  int rmax_a, rmax_b;                // largest ra, rb over directions
  int tc;                            // slab restores on the tensor cores: 1 3xTF32, 2 BF16x3
  int tc_single;                     // 1: single TF32 products instead of 3xTF32 (tc == 1, pre-pass)
  // large y-z planes (persistent yz kernel, slabs in global scratch)
  int large;                         // set by plan_yz
  long long slot_elems;              // scratch elements per block (set by plan_yz)
  int large_grid;                    // blocks of the persistent kernel
  void* slab_scratch;                // large_grid * slot_elems elements
  int n_stages;                      // pre-pass launches, in order
  GemmStage stages[kMaxGemmStages];
  int* status;                       // device status word
  cudaEvent_t* events;               // FMMFFT_NUM_STAGES + 1 events, or null
  cudaStream_t stream;
  // the restore pre-pass runs on `side`, overlapped with the forward x pass,
  // when side and both events are given and no stage events are recorded
  cudaStream_t side;
  cudaEvent_t fork, join;
  // schedule knobs (fmmfft_autotune); 0 = default
  int xrows;                         // x-pass rows per block as a multiple of the
                                     // lines one block iteration covers (1, 2, 4)
  int no_overlap;                    // 1: pre-pass in line with the x pass
  int tc_gemm;                       // pre-pass products on the tensor cores: 1 3xTF32, 2 BF16x3
  // box occupancy (Sec. II.A: empty boxes carry no sources and no testing
  // functions), device bytes, or null for a full grid: occ[v] per box
  // (v = (z Ky + y) Kx + x), rowocc[z Ky + y] per x-line (any box occupied)
  const unsigned char* occ = nullptr;
  const unsigned char* rowocc = nullptr;
  // when set, the inverse x pass is replaced by the fused inverse x pass +
  // disaggregation (Eq. 6) with these patterns / weights / output; s_out is
  // then not written.  Whole-plan launches only (p0 = 0, nw = 0).
  const XDisArgs* dis = nullptr;
  // direction block of this launch: directions p0 .. p0 + nw - 1 (nw = 0: all),
  // fields and intermediate addressed at their place in the full arrays; the
  // restore pre-pass runs only when `prepass` is set (it covers every direction)
  int p0 = 0, nw = 0;
  bool prepass = true;
};

// A translation schedule: the choices fmmfft_autotune makes for a plan.
struct Schedule {
  int xrows = 0;          // 0: default (2), else 1, 2 or 4
  int tc_slab = -1;       // -1: default (tensor cores when they apply), 0 off, 1 on
  int tc_gemm = -1;       // -1: default (tensor cores for 3xTF32 plans), 0 off, 1 on
  int no_overlap = 0;
};

// Kernel launchers (translate_launch.cu).  Return a cudaError_t.
cudaError_t launch_translate(const TranslateArgs& a);
// Largest shared-memory request of the yz kernel for the given args (bytes);
// 0 if the sizes are not supported by the compiled kernels.
size_t yz_smem_bytes(const TranslateArgs& a);
bool translate_supported(const TranslateArgs& a);
// Choose the yz kernel for the args: the fused one when its shared memory
// fits, else the large-plane one; sets a.large and a.slot_elems.  False when
// neither fits.
bool plan_yz(TranslateArgs& a);
// Tensor-core arithmetic of a precision: 1 3xTF32, 2 BF16x3, 0 none.
int tc_kind(int precision);
// Whether the slab restores of these args can run on the tensor cores.
bool tc_restore_applies(const TranslateArgs& a);

// Translation of a compressed plan with a caller-provided intermediate buffer
// (fmmfft_api.cpp), used by the allocation-free entry point.
// translate_scratch_bytes validates the plan and nrhs and returns the bytes of
// intermediate one call needs; translate_into validates the field buffers and
// launches the translation with `scratch` (scratch_bytes long) as intermediate.
int translate_scratch_bytes(fmmfft_plan p, int nrhs, size_t* bytes);
int translate_into(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* stream,
                   void* scratch, size_t scratch_bytes);
// The plan's own intermediate for nrhs RHS, allocated (after synchronising
// `stream`) when it is smaller; outputs its address and size.
int plan_intermediate(fmmfft_plan p, int nrhs, void* stream, void** inter, size_t* bytes);
// Stream that fmmfft_poll_status synchronises for this plan.
void plan_set_last_stream(fmmfft_plan p, void* stream);

// Arguments of one translation of plan p (the checks of fmmfft_translate,
// with `scratch` as the intermediate), without launching anything
// (fmmfft_api.cpp).
int translate_args_for(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* scratch, size_t scratch_bytes,
                       TranslateArgs* out);

// Shared launches of a batch (batch_launch.cu).  BatchDev: the batch's
// device descriptor buffer and the host copy of what it holds.
struct BatchDev {
  void* d_desc = nullptr;
  size_t bytes = 0;
  std::vector<unsigned char> host;
  std::vector<const void*> gemm_src;
  cudaEvent_t pre = nullptr;           // the merged pre-pass is done
};
// Whether a translation can join the batch's shared launches: complex64,
// y-z planes of the fused yz kernel (not the large-plane one), whole-plan
// launch.
bool batch_persistent_ok(const TranslateArgs& a);
// All translations of `args` grouped into shape classes (FFT extents,
// operator kind, restore arithmetic): the merged restore pre-pass on stream
// s, then per class one launch per phase (x forward, yz, x
// inverse) on lanes[class % lanes.size()] (streams already forked from s),
// so that classes overlap.  Uploads the descriptors to dev when they
// changed, after synchronising s and the lanes.
cudaError_t launch_translate_batch(const std::vector<TranslateArgs>& args, BatchDev& dev, cudaStream_t s,
                                   const std::vector<cudaStream_t>& lanes);
void batch_dev_release(BatchDev& dev);

// Aggregation (Eq. 4) and disaggregation (Eq. 6), farfield.cu.  P: patterns
// [n_dir][2][nb][V]; aggregation reads `in` = coefficients [nrhs][nb][V] and
// writes `out` = spectra [n_dir][2][nrhs][V]; disaggregation reads `in` =
// spectra and the weights w (n_dir doubles) and writes `out` = [nrhs][nb][V].
// Complex64 (float2) or, with fp64, complex128 (double2) elements.
struct FarFieldArgs {
  const void* P = nullptr;
  const void* in = nullptr;
  void* out = nullptr;
  const double* w = nullptr;
  int64_t V = 0;
  int nb = 0, nrhs = 0, n_dir = 0;
  bool fp64 = false;
  cudaStream_t stream = nullptr;
};
constexpr int kFarFieldMaxNb = 48;   // basis functions per box

// The inverse x pass fused with the disaggregation (Eq. 5's last DFT, then
// Eq. 6): reads the translated x-spectra `inter` ([F][n1][Ky Kz], F =
// n_dir 2 nrhs fields in the translation's order) and the patterns P, writes
// y = [nrhs][nb][V]; the translated fields themselves are never stored.
struct XDisArgs {
  const void* inter = nullptr;
  const void* P = nullptr;
  const double* w = nullptr;       // n_dir quadrature weights (device)
  void* y = nullptr;
  const void* tw = nullptr;        // W_n1^m, m < n1
  const unsigned char* occ = nullptr;      // box occupancy or null (TranslateArgs)
  const unsigned char* rowocc = nullptr;
  int n1 = 0, Kx = 0, rows = 0;    // rows = Ky Kz
  int nb = 0, nrhs = 0, n_dir = 0;
  bool fp64 = false;
  cudaStream_t stream = nullptr;
};
cudaError_t launch_xinv_disaggregate(const XDisArgs& a);
size_t aggregate_smem_bytes(int nb, bool fp64);
cudaError_t launch_aggregate(const FarFieldArgs& a);
cudaError_t launch_disaggregate(const FarFieldArgs& a);

}  // namespace fmm
