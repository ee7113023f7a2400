// Launch sequence of one translation: [restore pre-pass] -> xfwd -> yz -> xinv.
#include <cstring>

#include "translate_kernels.cuh"

namespace fmm {

#define FMM_YZ_DECL(TAG, F)                                                                  \
  cudaError_t launch_yz_##TAG##_##F(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, \
                                    cudaStream_t s);
FMM_YZ_DECL(f32, 0)
FMM_YZ_DECL(f32, 1)
FMM_YZ_DECL(f32, 2)
FMM_YZ_DECL(f64, 0)
FMM_YZ_DECL(f64, 1)
FMM_YZ_DECL(f64, 2)
#undef FMM_YZ_DECL
#define FMM_YZB_DECL(TAG, F)                                                                       \
  cudaError_t launch_yz_batch_##TAG##_##F(const YZParams& P, int n2, int n3, size_t smem, cudaStream_t s, \
                                          const BatchYZ* inst, int ninst, long long total);
FMM_YZB_DECL(f32, 0)
FMM_YZB_DECL(f32, 1)
FMM_YZB_DECL(f32, 2)
#undef FMM_YZB_DECL
#define FMM_YZL_DECL(TAG, F)                                                                  \
  cudaError_t launch_yzl_##TAG##_##F(const YZParams& P, int n2, int n3, dim3 grid, size_t smem, \
                                     cudaStream_t s);
FMM_YZL_DECL(f32, 0)
FMM_YZL_DECL(f32, 1)
FMM_YZL_DECL(f32, 2)
FMM_YZL_DECL(f64, 0)
FMM_YZL_DECL(f64, 1)
FMM_YZL_DECL(f64, 2)
#undef FMM_YZL_DECL

static const size_t kMaxSmem = 227 * 1024;

template <typename R, int N1>
static cudaError_t launch_x_inst(bool fwd, XPassParams P, int F, cudaStream_t s) {
  static std::atomic<int> optin_f[kMaxDevices], optin_i[kMaxDevices];
  P.rows_per_block = xpass_rows_per_block<R, N1>(P.rows, P.rows_per_block);
  const size_t smem =
      xpass_smem<R, N1>(P.rows_per_block) + (P.occ && P.rowocc ? xpass_mask_bytes(P.rows_per_block, P.Kx) : 0);
  dim3 grid((unsigned)(((P.rows + P.rows_per_block - 1) / P.rows_per_block) * (size_t)F));
  if (fwd) {
    cudaError_t e = smem_optin((const void*)xfwd_kernel<R, N1>, optin_f);
    if (e != cudaSuccess) return e;
    xfwd_kernel<R, N1><<<grid, kThreads, smem, s>>>(P);
  } else {
    cudaError_t e = smem_optin((const void*)xinv_kernel<R, N1>, optin_i);
    if (e != cudaSuccess) return e;
    xinv_kernel<R, N1><<<grid, kThreads, smem, s>>>(P);
  }
  return cudaGetLastError();
}

// Batch mode of the x passes over the `total` items of the table's instances
// with this n1 (float), one item per block.
template <int N1>
static cudaError_t launch_x_batch_inst(bool fwd, const BatchXTable& T, long long total, size_t smem,
                                       cudaStream_t s) {
  static std::atomic<int> optin_f[kMaxDevices], optin_i[kMaxDevices];
  if (total > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (fwd) {
    auto kern = xfwd_batch_kernel<float, N1>;
    cudaError_t e = smem_optin((const void*)kern, optin_f);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)total, kThreads, smem, s>>>(T);
  } else {
    auto kern = xinv_batch_kernel<float, N1>;
    cudaError_t e = smem_optin((const void*)kern, optin_i);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)total, kThreads, smem, s>>>(T);
  }
  return cudaGetLastError();
}

cudaError_t launch_x_batch(bool fwd, int n1, const BatchXTable& T, long long total, size_t smem, cudaStream_t s) {
  switch (n1) {
    case 4: return launch_x_batch_inst<4>(fwd, T, total, smem, s);
    case 8: return launch_x_batch_inst<8>(fwd, T, total, smem, s);
    case 16: return launch_x_batch_inst<16>(fwd, T, total, smem, s);
    case 32: return launch_x_batch_inst<32>(fwd, T, total, smem, s);
    case 64: return launch_x_batch_inst<64>(fwd, T, total, smem, s);
    case 128: return launch_x_batch_inst<128>(fwd, T, total, smem, s);
    case 256: return launch_x_batch_inst<256>(fwd, T, total, smem, s);
    default: return cudaErrorInvalidValue;
  }
}

// x-pass rows per block and shared memory of an n1 (float), as a single
// translation chooses them.
void x_pass_shape(int n1, int rows, int mult, int* rpb, size_t* smem) {
  switch (n1) {
#define FMM_XSHAPE(N)                                   \
    case N:                                             \
      *rpb = xpass_rows_per_block<float, N>(rows, mult); \
      *smem = xpass_smem<float, N>(*rpb);               \
      return;
    FMM_XSHAPE(4) FMM_XSHAPE(8) FMM_XSHAPE(16) FMM_XSHAPE(32) FMM_XSHAPE(64) FMM_XSHAPE(128) FMM_XSHAPE(256)
#undef FMM_XSHAPE
    default:
      *rpb = 0;
      *smem = 0;
  }
}

cudaError_t launch_yz_batch(int fmt, const YZParams& P, int n2, int n3, size_t smem, cudaStream_t s,
                            const BatchYZ* inst, int ninst, long long total) {
  switch (fmt) {
    case 0: return launch_yz_batch_f32_0(P, n2, n3, smem, s, inst, ninst, total);
    case 1: return launch_yz_batch_f32_1(P, n2, n3, smem, s, inst, ninst, total);
    case 2: return launch_yz_batch_f32_2(P, n2, n3, smem, s, inst, ninst, total);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
static cudaError_t launch_x(bool fwd, int n1, const XPassParams& P, int F, cudaStream_t s) {
  switch (n1) {
    case 4: return launch_x_inst<R, 4>(fwd, P, F, s);
    case 8: return launch_x_inst<R, 8>(fwd, P, F, s);
    case 16: return launch_x_inst<R, 16>(fwd, P, F, s);
    case 32: return launch_x_inst<R, 32>(fwd, P, F, s);
    case 64: return launch_x_inst<R, 64>(fwd, P, F, s);
    case 128: return launch_x_inst<R, 128>(fwd, P, F, s);
    case 256: return launch_x_inst<R, 256>(fwd, P, F, s);
    default: return cudaErrorInvalidValue;
  }
}

static bool pow2_in(int n, int lo, int hi) { return n >= lo && n <= hi && (n & (n - 1)) == 0; }

template <typename R, int N2>
static size_t yz_smem_n3(int n3, int fmt, int ra, int rb, bool tc) {
  switch (n3) {
    case 4: return YZLayout<R, N2, 4>::smem_bytes(fmt, ra, rb, tc);
    case 8: return YZLayout<R, N2, 8>::smem_bytes(fmt, ra, rb, tc);
    case 16: return YZLayout<R, N2, 16>::smem_bytes(fmt, ra, rb, tc);
    case 32: return YZLayout<R, N2, 32>::smem_bytes(fmt, ra, rb, tc);
    case 64: return YZLayout<R, N2, 64>::smem_bytes(fmt, ra, rb, tc);
    case 128: return YZLayout<R, N2, 128>::smem_bytes(fmt, ra, rb, tc);
    default: return 0;
  }
}

template <typename R>
static size_t yz_smem_any(int n2, int n3, int fmt, int ra, int rb, bool tc) {
  switch (n2) {
    case 4: return yz_smem_n3<R, 4>(n3, fmt, ra, rb, tc);
    case 8: return yz_smem_n3<R, 8>(n3, fmt, ra, rb, tc);
    case 16: return yz_smem_n3<R, 16>(n3, fmt, ra, rb, tc);
    case 32: return yz_smem_n3<R, 32>(n3, fmt, ra, rb, tc);
    case 64: return yz_smem_n3<R, 64>(n3, fmt, ra, rb, tc);
    case 128: return yz_smem_n3<R, 128>(n3, fmt, ra, rb, tc);
    default: return 0;
  }
}

int tc_kind(int precision) {
  return (precision == FMMFFT_PREC_C64_3XTF32 || precision == FMMFFT_PREC_C64_TF32)
             ? 1
             : (precision == FMMFFT_PREC_C64_BF16X3 ? 2 : 0);
}

bool tc_restore_applies(const TranslateArgs& a) {
  const bool tiles = (a.n[1] % 64 == 0 && a.n[2] % 64 == 0) ||
                     (a.n[1] % 32 == 0 && a.n[2] % 32 == 0 && a.n[1] <= 64 && a.n[2] <= 64);
  return tc_kind(a.precision) != 0 && a.yz_fmt != 0 && tiles &&
         (a.yz_fmt == 2 || a.rmax_b <= 64);
}

template <typename R>
static bool yzl_shape(int n2, int n3, int fmt, bool tc, int rb, size_t* smem, long long* slot) {
#define FMM_YZL_SHAPE(A, B)                                    \
  if (n2 == A && n3 == B) {                                    \
    *smem = YZLLayout<R, A, B>::smem_bytes(fmt, tc);           \
    *slot = YZLLayout<R, A, B>::slot_elems(fmt, rb);           \
    return true;                                               \
  }
  FMM_YZL_SHAPE(128, 128)
  FMM_YZL_SHAPE(256, 64)
  FMM_YZL_SHAPE(256, 128)
#undef FMM_YZL_SHAPE
  return false;
}

static size_t yzl_smem_bytes(const TranslateArgs& a, long long* slot) {
  size_t smem = 0;
  long long sl = 0;
  const bool ok = a.precision == FMMFFT_PREC_C128
                      ? yzl_shape<double>(a.n[1], a.n[2], a.yz_fmt, false, a.rmax_b, &smem, &sl)
                      : yzl_shape<float>(a.n[1], a.n[2], a.yz_fmt, a.tc != 0, a.rmax_b, &smem, &sl);
  if (slot) *slot = sl;
  return ok ? smem : 0;
}

static size_t yz_fused_smem_bytes(const TranslateArgs& a) {
  const bool tc = a.tc != 0;
  if (a.n[1] > 128) return 0;
  return a.precision == FMMFFT_PREC_C128
             ? yz_smem_any<double>(a.n[1], a.n[2], a.yz_fmt, a.rmax_a, a.rmax_b, false)
             : yz_smem_any<float>(a.n[1], a.n[2], a.yz_fmt, a.rmax_a, a.rmax_b, tc);
}

bool plan_yz(TranslateArgs& a) {
  a.large = 0;
  a.slot_elems = 0;
  const size_t fused = yz_fused_smem_bytes(a);
  if (fused != 0 && fused <= kMaxSmem) return true;
  long long slot = 0;
  const size_t large = yzl_smem_bytes(a, &slot);
  if (large == 0 || large > kMaxSmem) return false;
  a.large = 1;
  a.slot_elems = slot;
  return true;
}

size_t yz_smem_bytes(const TranslateArgs& a) {
  return a.large ? yzl_smem_bytes(a, nullptr) : yz_fused_smem_bytes(a);
}

bool translate_supported(const TranslateArgs& a) {
  if (!pow2_in(a.n[0], 4, 256) || !pow2_in(a.n[1], 4, 256) || !pow2_in(a.n[2], 4, 128)) return false;
  if (a.yz_fmt < 0 || a.yz_fmt > 2) return false;
  TranslateArgs b = a;
  // x-pass shared memory at the largest rows-per-block candidate is bounded
  // by construction (<= 96 KB)
  return plan_yz(b);
}

static cudaError_t launch_yz(const TranslateArgs& a, const YZParams& Y, dim3 grid, size_t smem) {
  const int n2 = a.n[1], n3 = a.n[2];
  if (a.large) {
    if (a.precision == FMMFFT_PREC_C128) {
      switch (a.yz_fmt) {
        case 0: return launch_yzl_f64_0(Y, n2, n3, grid, smem, a.stream);
        case 1: return launch_yzl_f64_1(Y, n2, n3, grid, smem, a.stream);
        case 2: return launch_yzl_f64_2(Y, n2, n3, grid, smem, a.stream);
        default: return cudaErrorInvalidValue;
      }
    }
    switch (a.yz_fmt) {
      case 0: return launch_yzl_f32_0(Y, n2, n3, grid, smem, a.stream);
      case 1: return launch_yzl_f32_1(Y, n2, n3, grid, smem, a.stream);
      case 2: return launch_yzl_f32_2(Y, n2, n3, grid, smem, a.stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (a.precision == FMMFFT_PREC_C128) {
    switch (a.yz_fmt) {
      case 0: return launch_yz_f64_0(Y, n2, n3, grid, smem, a.stream);
      case 1: return launch_yz_f64_1(Y, n2, n3, grid, smem, a.stream);
      case 2: return launch_yz_f64_2(Y, n2, n3, grid, smem, a.stream);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (a.yz_fmt) {
    case 0: return launch_yz_f32_0(Y, n2, n3, grid, smem, a.stream);
    case 1: return launch_yz_f32_1(Y, n2, n3, grid, smem, a.stream);
    case 2: return launch_yz_f32_2(Y, n2, n3, grid, smem, a.stream);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
static cudaError_t launch_all(const TranslateArgs& a) {
  const int nw = a.nw > 0 ? a.nw : a.n_dir;
  if (a.p0 < 0 || a.p0 + nw > a.n_dir) return cudaErrorInvalidValue;
  const int F = nw * 2 * a.nrhs;
  const size_t f0 = (size_t)a.p0 * 2 * a.nrhs;     // first field of the block
  const int rows = a.K[1] * a.K[2];
  const size_t es = sizeof(cx<R>);
  cudaError_t e;
  auto mark = [&](int i) {
    if (a.events) cudaEventRecord(a.events[i], a.stream);
  };
  mark(0);
  // the pre-pass needs only the stored factors: overlap it with the forward
  // x pass on the side stream (serially when stage times are recorded)
  const int n_stages = a.prepass ? a.n_stages : 0;
  const bool overlap = n_stages > 0 && a.side && a.fork && a.join && !a.events && !a.no_overlap;
  cudaStream_t ps = a.stream;
  if (overlap) {
    if ((e = cudaEventRecord(a.fork, a.stream)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(a.side, a.fork, 0)) != cudaSuccess) return e;
    ps = a.side;
  }
  // 3xTF32 plans run the pre-pass products on the tensor cores too
  const bool tc_gemm = a.tc_gemm != 0;
  if (tc_gemm) {
    static std::atomic<int> optin_t[kMaxDevices], optin_b[kMaxDevices];
    e = smem_optin((const void*)cgemm_batched_tc_kernel<false>, optin_t);
    if (e == cudaSuccess) e = smem_optin((const void*)cgemm_batched_tc_kernel<true>, optin_b);
    if (e != cudaSuccess) return e;
  }
  for (int i = 0; i < n_stages; ++i) {
    const GemmStage& g = a.stages[i];
    dim3 grid((g.max_n + kGemmT - 1) / kGemmT, (g.max_m + kGemmT - 1) / kGemmT, g.batch);
    if (tc_gemm && sizeof(R) == 4 && a.tc_gemm == 2)
      cgemm_batched_tc_kernel<true><<<grid, kThreads, kTcGemmSmem, ps>>>(g.desc, a.status, 0);
    else if (tc_gemm && sizeof(R) == 4)
      cgemm_batched_tc_kernel<false><<<grid, kThreads, kTcGemmSmem, ps>>>(g.desc, a.status, a.tc_single);
    else cgemm_batched_kernel<R><<<grid, kThreads, 0, ps>>>(g.desc);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if (overlap && (e = cudaEventRecord(a.join, a.side)) != cudaSuccess) return e;
  mark(1);
  XPassParams X;
  X.src = (const char*)a.s_in + f0 * a.K[0] * rows * es;
  X.dst = (char*)a.inter + f0 * a.n[0] * rows * es;
  X.tw = a.tw[0];
  X.Kx = a.K[0];
  X.rows = rows;
  X.rows_per_block = a.xrows;   // multiplier in, rows per block chosen per launch
  X.occ = a.occ;
  X.rowocc = a.rowocc;
  if ((e = launch_x<R>(true, a.n[0], X, F, a.stream)) != cudaSuccess) return e;
  if (overlap && (e = cudaStreamWaitEvent(a.stream, a.join, 0)) != cudaSuccess) return e;
  mark(2);

  YZParams Y;
  Y.inter = a.inter;
  Y.tw2 = a.tw[1];
  Y.tw3 = a.tw[2];
  Y.Ky = a.K[1];
  Y.Kz = a.K[2];
  Y.n1 = a.n[0];
  Y.nf = 2 * a.nrhs;
  Y.op = a.op_plain;
  Y.desc = a.slab;
  Y.scale = 1.0 / ((double)a.n[0] * a.n[1] * a.n[2]);
  Y.rmax_a = a.rmax_a;
  Y.rmax_b = a.rmax_b;
  Y.status = a.status;
  Y.tc = a.tc;
  Y.tc_single = a.tc_single;
  Y.n_dir = nw;
  Y.p0 = a.p0;
  Y.slab_scratch = a.slab_scratch;
  Y.slot_elems = a.slot_elems;
  const size_t smem = yz_smem_bytes(a);
  if (a.large && a.yz_fmt != 0 && !a.slab_scratch) return cudaErrorInvalidValue;
  const int items = a.n[0] * nw;
  dim3 grid = a.large ? dim3((unsigned)(items < a.large_grid ? items : a.large_grid)) : dim3(a.n[0], nw);
  if ((e = launch_yz(a, Y, grid, smem)) != cudaSuccess) return e;
  mark(3);

  if (a.dis) {
    if (a.p0 != 0 || nw != a.n_dir) return cudaErrorInvalidValue;
    XDisArgs d = *a.dis;
    d.inter = a.inter;
    d.tw = a.tw[0];
    d.occ = a.occ;
    d.rowocc = a.rowocc;
    d.n1 = a.n[0];
    d.Kx = a.K[0];
    d.rows = rows;
    d.nrhs = a.nrhs;
    d.n_dir = a.n_dir;
    d.fp64 = sizeof(R) == 8;
    d.stream = a.stream;
    e = launch_xinv_disaggregate(d);
    mark(4);
    return e;
  }
  X.src = (const char*)a.inter + f0 * a.n[0] * rows * es;
  X.dst = (char*)a.s_out + f0 * a.K[0] * rows * es;
  e = launch_x<R>(false, a.n[0], X, F, a.stream);
  mark(4);
  return e;
}

cudaError_t launch_translate(const TranslateArgs& a) {
  return a.precision == FMMFFT_PREC_C128 ? launch_all<double>(a) : launch_all<float>(a);
}

}  // namespace fmm
