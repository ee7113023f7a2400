// Launch sequence of one translation: [restore step 1] -> xfwd -> yz -> xinv.
#include "translate_kernels.cuh"

namespace fmm {

cudaError_t launch_yz_f32(const YZParams& P, int n2, int n3, int fmt, dim3 grid, size_t smem,
                          cudaStream_t s);
size_t yz_smem_f32(int n2, int n3, int fmt, int r2, int r3, int variant);
cudaError_t launch_yz_f64(const YZParams& P, int n2, int n3, int fmt, dim3 grid, size_t smem,
                          cudaStream_t s);
size_t yz_smem_f64(int n2, int n3, int fmt, int r2, int r3, int variant);

static const size_t kMaxSmem = 227 * 1024;
static const int kHCols = 128;

template <typename R, int N1>
static int xpass_rows_per_block(int rows) {
  int rpb = 2 * Line<N1>::LPI;
  while (rpb > Line<N1>::LPI && xpass_smem<R, N1>(rpb) > 96 * 1024) rpb /= 2;
  return rpb < rows ? rpb : rows;
}

template <typename R, int N1>
static cudaError_t launch_x_inst(bool fwd, XPassParams P, int F, cudaStream_t s) {
  static size_t configured_f = 0, configured_i = 0;
  P.rows_per_block = xpass_rows_per_block<R, N1>(P.rows);
  const size_t smem = xpass_smem<R, N1>(P.rows_per_block);
  dim3 grid((unsigned)(((P.rows + P.rows_per_block - 1) / P.rows_per_block) * (size_t)F));
  if (fwd) {
    if (smem > configured_f) {
      cudaError_t e = cudaFuncSetAttribute(xfwd_kernel<R, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured_f = smem;
    }
    xfwd_kernel<R, N1><<<grid, kThreads, smem, s>>>(P);
  } else {
    if (smem > configured_i) {
      cudaError_t e = cudaFuncSetAttribute(xinv_kernel<R, N1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured_i = smem;
    }
    xinv_kernel<R, N1><<<grid, kThreads, smem, s>>>(P);
  }
  return cudaGetLastError();
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

size_t yz_smem_bytes(const TranslateArgs& a) {
  const int fmt = (a.format == FMMFFT_FORMAT_NONE) ? 0 : 1;
  const int r2 = a.t3_rmax[1], r3 = a.t3_rmax[2];
  return a.precision == FMMFFT_PREC_C128 ? yz_smem_f64(a.n[1], a.n[2], fmt, r2, r3, a.yz_variant)
                                         : yz_smem_f32(a.n[1], a.n[2], fmt, r2, r3, a.yz_variant);
}

static size_t h_smem_bytes(const TranslateArgs& a) {
  const size_t es = a.precision == FMMFFT_PREC_C128 ? 16 : 8;
  return es * ((size_t)a.n[0] * a.t3_rmax[0] + (size_t)a.t3_rmax[0] * kHCols);
}

bool translate_supported(const TranslateArgs& a) {
  if (!pow2_in(a.n[0], 4, 256) || !pow2_in(a.n[1], 4, 128) || !pow2_in(a.n[2], 4, 128)) return false;
  if (a.format != FMMFFT_FORMAT_NONE &&
      !(a.format == FMMFFT_FORMAT_3D && a.decomp == FMMFFT_DECOMP_TUCKER))
    return false;
  const size_t s = yz_smem_bytes(a);
  if (s == 0 || s > kMaxSmem) return false;
  if (a.format != FMMFFT_FORMAT_NONE && h_smem_bytes(a) > kMaxSmem) return false;
  // x-pass shared memory at the largest rows-per-block candidate is bounded
  // by construction (<= 96 KB)
  return true;
}

template <typename R>
static cudaError_t launch_all(const TranslateArgs& a) {
  const int F = a.n_dir * 2 * a.nrhs;
  const int rows = a.K[1] * a.K[2];
  cudaError_t e;
  const bool tucker = a.format == FMMFFT_FORMAT_3D && a.decomp == FMMFFT_DECOMP_TUCKER;
  auto mark = [&](int i) {
    if (a.events) cudaEventRecord(a.events[i], a.stream);
  };
  mark(0);
  if (tucker) {
    HParams H;
    H.desc = a.t3_desc;
    H.pack = a.t3_pack;
    H.hbuf = a.t3_h;
    H.n1 = a.n[0];
    H.cols_per_block = kHCols;
    H.rmax1 = a.t3_rmax[0];
    H.status = a.status;
    const size_t smem = h_smem_bytes(a);
    static size_t configured = 0;
    if (smem > configured) {
      e = cudaFuncSetAttribute(tucker3d_h_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      configured = smem;
    }
    const int maxcols = a.t3_rmax[1] * a.t3_rmax[2];
    dim3 grid((maxcols + kHCols - 1) / kHCols, a.n_dir);
    tucker3d_h_kernel<R><<<grid, kThreads, smem, a.stream>>>(H);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  mark(1);
  XPassParams X;
  X.src = a.s_in;
  X.dst = a.inter;
  X.tw = a.tw[0];
  X.Kx = a.K[0];
  X.rows = rows;
  X.rows_per_block = 0;
  if ((e = launch_x<R>(true, a.n[0], X, F, a.stream)) != cudaSuccess) return e;
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
  Y.desc = a.t3_desc;
  Y.pack = a.t3_pack;
  Y.hbuf = a.t3_h;
  Y.scale = 1.0 / ((double)a.n[0] * a.n[1] * a.n[2]);
  Y.rmax2 = a.t3_rmax[1];
  Y.rmax3 = a.t3_rmax[2];
  Y.status = a.status;
  Y.variant = a.yz_variant;
  const int fmt = tucker ? 1 : 0;
  const size_t smem = yz_smem_bytes(a);
  dim3 grid(a.n[0], a.n_dir);
  e = (a.precision == FMMFFT_PREC_C128)
          ? launch_yz_f64(Y, a.n[1], a.n[2], fmt, grid, smem, a.stream)
          : launch_yz_f32(Y, a.n[1], a.n[2], fmt, grid, smem, a.stream);
  if (e != cudaSuccess) return e;
  mark(3);

  X.src = a.inter;
  X.dst = a.s_out;
  e = launch_x<R>(false, a.n[0], X, F, a.stream);
  mark(4);
  return e;
}

cudaError_t launch_translate(const TranslateArgs& a) {
  return a.precision == FMMFFT_PREC_C128 ? launch_all<double>(a) : launch_all<float>(a);
}

}  // namespace fmm
