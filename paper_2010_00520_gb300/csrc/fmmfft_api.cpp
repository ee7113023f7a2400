// C ABI of the translation library: plan life cycle, set-up, translation.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <sstream>
#include <string>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/fmmfft.h"
#include "host_decomp.h"
#include "host_setup.h"
#include "plan_internal.h"
#include "plan_layout.h"

using fmm::cdouble;

constexpr int kHostBlocksMax = 64;     // direction blocks of the host pipeline
constexpr int kHostBlocksDefault = 12;

struct fmmfft_plan_s {
  int K[3] = {0, 0, 0};
  int n[3] = {0, 0, 0};
  int L = 0;
  double a = 0, k0 = 0, tol = 0;
  int format = 0, decomp = 0;
  int precision = FMMFFT_PREC_C64;
  int nphi_rule = 0, near_rule = 0, prefactor = 0, trunc_rule = 0;
  double kappa = 4.0;
  double eps_re = 1.0, eps_im = 0.0;   // relative permittivity of the medium
  int dir_first = 0, dir_count = 0;    // direction block of a shard plan (count 0: to the end)
  int n_dir_grid = 0;                  // directions of the whole grid
  int n_dir = 0;                       // directions of this plan
  std::vector<double> khat, weights;
  bool ready = false;
  // device state
  void* d_tw[3] = {nullptr, nullptr, nullptr};
  void* d_op = nullptr;         // format NONE: T~_p / (n1 n2 n3), [p][x][z][y]
                                //   ([p][x][y][z] for the large-plane yz kernel)
  void* d_pack = nullptr;       // compressed formats: stored factors
  void* d_scratch = nullptr;    // compressed formats: restore pre-pass outputs
  fmm::SlabDesc* d_slab = nullptr;
  fmm::GemmDesc* d_gemm = nullptr;
  fmm::GemmStage stages[fmm::kMaxGemmStages] = {};
  int n_stages = 0;
  int yz_fmt = 0;
  int rmax_a = 0, rmax_b = 0;
  void* d_slabs = nullptr;      // large planes: per-block slab slots
  size_t slabs_bytes = 0;
  int large_grid = 0;           // blocks of the persistent large-plane kernel
  void* d_inter = nullptr;
  void* d_weights = nullptr;   // quadrature weights on the device (far-field steps)
  void* d_occ = nullptr;       // box occupancy (V bytes) then x-line occupancy (Ky Kz bytes)
  bool occ_set = false;        // a mask is in force (d_occ stays allocated once made)
  size_t inter_bytes = 0;
  void* d_io = nullptr;       // device copies for fmmfft_translate_host
  size_t io_bytes = 0;
  int* d_status = nullptr;
  cudaStream_t last_stream = nullptr;
  cudaStream_t side = nullptr;  // restore pre-pass, overlapped with the x pass
  cudaEvent_t fork = nullptr, join = nullptr;
  // copy/compute pipeline of fmmfft_translate_host: copy streams, events
  // (start, done, then one in / out pair per direction block) and block count
  cudaStream_t h2d = nullptr, d2h = nullptr;
  cudaEvent_t hev[2 + 2 * kHostBlocksMax] = {};
  int host_blocks = 0;          // FMMFFT_KEY_HOST_BLOCKS, 0: default
  fmm::Schedule sched;          // fmmfft_autotune's choices
  bool profile = false;
  bool profiled_run = false;
  bool measure_err = false;     // FMMFFT_KEY_RESTORE_ERROR
  double restore_err = -1.0;    // FP64 restore error of the set-up, -1: not measured
  cudaEvent_t events[FMMFFT_NUM_STAGES + 1] = {};
  // host-side bookkeeping
  std::vector<int> ranks3;      // 3D formats: n_dir x 3
  int rmax[6] = {0, 0, 0, 0, 0, 0};
  double mean_rank[3] = {0, 0, 0};
  int64_t elements_plain = 0, elements_compressed = 0;
  int64_t bytes_operator = 0, bytes_restore = 0;
  double setup_seconds = 0;
  fmm::Layout layout;           // host copy of the compressed store (plan save)
};

namespace {

int embed_extent(int K) {
  int n = 1;
  while (n < 2 * K - 1) n *= 2;
  return n < 2 ? 2 : n;
}

size_t elem_bytes(const fmmfft_plan_s* p) { return p->precision == FMMFFT_PREC_C128 ? 16 : 8; }

void free_dev(void*& ptr) {
  if (ptr) cudaFree(ptr);
  ptr = nullptr;
}

void release_operator(fmmfft_plan_s* p) {
  for (auto& t : p->d_tw) free_dev(t);
  free_dev(p->d_op);
  free_dev(p->d_pack);
  free_dev(p->d_scratch);
  void* d = p->d_slab;
  free_dev(d);
  p->d_slab = nullptr;
  d = p->d_gemm;
  free_dev(d);
  p->d_gemm = nullptr;
  p->n_stages = 0;
  free_dev(p->d_slabs);
  p->slabs_bytes = 0;
  p->ready = false;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return FMMFFT_OK;
  if (e == cudaErrorMemoryAllocation) return FMMFFT_ERR_OOM;
  return FMMFFT_ERR_CUDA;
}

int dev_alloc(void** ptr, size_t bytes) {
  cudaError_t e = cudaMalloc(ptr, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return cuda_status(e);
  }
  return FMMFFT_OK;
}

// host complex doubles -> device float2 / double2
int upload_complex(void** dst, const std::vector<cdouble>& src, bool dbl) {
  const size_t n = src.size();
  int st;
  if (dbl) {
    if ((st = dev_alloc(dst, n * 16)) != FMMFFT_OK) return st;
    return cuda_status(cudaMemcpy(*dst, src.data(), n * 16, cudaMemcpyHostToDevice));
  }
  std::vector<float> f(2 * n);
  for (size_t i = 0; i < n; ++i) {
    f[2 * i] = (float)src[i].real();
    f[2 * i + 1] = (float)src[i].imag();
  }
  if ((st = dev_alloc(dst, n * 8)) != FMMFFT_OK) return st;
  return cuda_status(cudaMemcpy(*dst, f.data(), n * 8, cudaMemcpyHostToDevice));
}

int ensure_common(fmmfft_plan_s* p) {
  const bool dbl = p->precision == FMMFFT_PREC_C128;
  for (int ax = 0; ax < 3; ++ax) {
    if (p->d_tw[ax]) continue;
    const int m = p->n[ax];
    std::vector<cdouble> tw(m);
    for (int k = 0; k < m; ++k) tw[k] = std::polar(1.0, -2.0 * 3.14159265358979323846 * k / m);
    int st = upload_complex(&p->d_tw[ax], tw, dbl);
    if (st != FMMFFT_OK) return st;
  }
  if (!p->side && p->format != FMMFFT_FORMAT_NONE) {
    if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return FMMFFT_ERR_CUDA;
    }
  }
  if (!p->d_status) {
    void* s = nullptr;
    int st = dev_alloc(&s, sizeof(int));
    if (st != FMMFFT_OK) return st;
    p->d_status = (int*)s;
    if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

// The plan's directions: the grid of Sec. II.A for its L and N_phi rule, cut
// to the block [dir_first, dir_first + dir_count) for a shard plan.
int set_directions(fmmfft_plan_s* p, int nphi_rule, int first, int count) {
  const int nphi = nphi_rule == 0 ? 2 * (p->L + 1) : 2 * p->L + 1;
  const int grid = (p->L + 1) * nphi;
  const int cnt = count == 0 ? grid - first : count;
  if (first < 0 || count < 0 || first >= grid || cnt < 1 || first + cnt > grid) return FMMFFT_ERR_INVALID_ARG;
  std::vector<double> kh, w;
  fmm::direction_grid(p->L, nphi, kh, w);
  p->khat.assign(kh.begin() + 3 * (size_t)first, kh.begin() + 3 * (size_t)(first + cnt));
  p->weights.assign(w.begin() + first, w.begin() + first + cnt);
  p->nphi_rule = nphi_rule;
  p->dir_first = first;
  p->dir_count = count;
  p->n_dir_grid = grid;
  p->n_dir = cnt;
  return FMMFFT_OK;
}

fmm::TranslateArgs base_args(const fmmfft_plan_s* p) {
  fmm::TranslateArgs a;
  std::memset(&a, 0, sizeof(a));
  for (int i = 0; i < 3; ++i) {
    a.K[i] = p->K[i];
    a.n[i] = p->n[i];
    a.tw[i] = p->d_tw[i];
  }
  a.n_dir = p->n_dir;
  a.precision = p->precision;
  a.yz_fmt = p->format == FMMFFT_FORMAT_NONE ? 0 : p->yz_fmt;
  a.op_plain = p->d_op;
  a.slab = p->d_slab;
  a.rmax_a = p->rmax_a;
  a.rmax_b = p->rmax_b;
  a.n_stages = p->n_stages;
  for (int i = 0; i < p->n_stages; ++i) a.stages[i] = p->stages[i];
  a.status = p->d_status;
  a.tc = fmm::tc_restore_applies(a) && p->sched.tc_slab != 0 ? fmm::tc_kind(p->precision) : 0;
  a.tc_single = p->precision == FMMFFT_PREC_C64_TF32 ? 1 : 0;
  a.tc_gemm = p->sched.tc_gemm != 0 ? fmm::tc_kind(p->precision) : 0;
  a.xrows = p->sched.xrows;
  a.no_overlap = p->sched.no_overlap;
  fmm::plan_yz(a);
  a.large_grid = p->large_grid;
  a.slab_scratch = p->d_slabs;
  a.side = p->side;
  a.fork = p->fork;
  a.join = p->join;
  a.p0 = 0;
  a.nw = 0;
  a.prepass = true;
  if (p->occ_set && p->d_occ) {
    a.occ = (const unsigned char*)p->d_occ;
    a.rowocc = a.occ + (size_t)p->K[0] * p->K[1] * p->K[2];
  }
  return a;
}

// Blocks of the persistent large-plane yz kernel: two per SM of the current
// device (its shared memory allows no more).
int query_large_grid(fmmfft_plan_s* p) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  p->large_grid = 2 * sms;
  return FMMFFT_OK;
}

// Slab slots of the large-plane kernel for a compressed plan that needs them.
int ensure_slabs(fmmfft_plan_s* p) {
  fmm::TranslateArgs a = base_args(p);
  if (!a.large || a.yz_fmt == 0) return FMMFFT_OK;
  const size_t bytes = (size_t)a.large_grid * (size_t)a.slot_elems * elem_bytes(p);
  if (bytes <= p->slabs_bytes && p->d_slabs) return FMMFFT_OK;
  free_dev(p->d_slabs);
  p->slabs_bytes = 0;
  int st = dev_alloc(&p->d_slabs, bytes);
  if (st != FMMFFT_OK) return st;
  p->slabs_bytes = bytes;
  return FMMFFT_OK;
}

// Plain store: T~_p scaled by 1/(n1 n2 n3), [p][x][z][y] for the fused yz
// kernel (rows copied into its shared-memory slab) or [p][x][y][z] for the
// large-plane one (read column by column from global memory).  `That` is
// indexed ((p n1 + x) n2 + y) n3 + z.
int upload_plain(fmmfft_plan_s* p, const std::function<const cdouble*(int)>& slab_of) {
  const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
  const size_t per = (size_t)n1 * n2 * n3;
  const double sc = 1.0 / (double)per;
  const bool by_column = base_args(p).large != 0;
  std::vector<cdouble> h(per * p->n_dir);
  fmm::parallel_for(p->n_dir, [&](int d) {
    const cdouble* T = slab_of(d);
    cdouble* o = &h[per * d];
    for (int x = 0; x < n1; ++x)
      for (int y = 0; y < n2; ++y)
        for (int z = 0; z < n3; ++z) {
          const size_t to = by_column ? ((size_t)x * n2 + y) * n3 + z : ((size_t)x * n3 + z) * n2 + y;
          o[to] = T[((size_t)x * n2 + y) * n3 + z] * sc;
        }
  });
  free_dev(p->d_op);
  int st = upload_complex(&p->d_op, h, p->precision == FMMFFT_PREC_C128);
  if (st != FMMFFT_OK) return st;
  p->elements_plain = (int64_t)per * p->n_dir;
  p->elements_compressed = p->elements_plain;
  p->bytes_operator = (int64_t)(per * p->n_dir * elem_bytes(p));
  for (int i = 0; i < 6; ++i) p->rmax[i] = 0;
  return FMMFFT_OK;
}

// Compressed store: factors, restore scratch and the descriptors of the
// restore schedule (pre-pass products and per-direction slab restores).
int upload_layout(fmmfft_plan_s* p, const fmm::Layout& L) {
  const bool dbl = p->precision == FMMFFT_PREC_C128;
  const size_t es = elem_bytes(p);
  if ((int)L.stages.size() > fmm::kMaxGemmStages) return FMMFFT_ERR_UNSUPPORTED;
  free_dev(p->d_pack);
  int st = upload_complex(&p->d_pack, L.pack, dbl);
  if (st != FMMFFT_OK) return st;
  free_dev(p->d_scratch);
  if ((st = dev_alloc(&p->d_scratch, (size_t)L.scratch * es)) != FMMFFT_OK) return st;
  std::vector<std::vector<fmm::GemmDesc>> g;
  fmm::bind_gemms(L, p->d_pack, p->d_scratch, es, g);
  std::vector<fmm::GemmDesc> flat;
  for (auto& stage : g) flat.insert(flat.end(), stage.begin(), stage.end());
  void* dg = nullptr;
  if ((st = dev_alloc(&dg, sizeof(fmm::GemmDesc) * std::max<size_t>(flat.size(), 1))) != FMMFFT_OK) return st;
  p->d_gemm = (fmm::GemmDesc*)dg;
  if (!flat.empty() &&
      cudaMemcpy(dg, flat.data(), sizeof(fmm::GemmDesc) * flat.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return FMMFFT_ERR_CUDA;
  p->n_stages = (int)g.size();
  size_t at = 0;
  for (int i = 0; i < p->n_stages; ++i) {
    fmm::GemmStage& S = p->stages[i];
    S.desc = p->d_gemm + at;
    S.batch = (int)g[i].size();
    S.max_m = 0;
    S.max_n = 0;
    for (auto& d : g[i]) {
      S.max_m = std::max(S.max_m, d.M);
      S.max_n = std::max(S.max_n, d.N);
    }
    at += g[i].size();
  }
  std::vector<fmm::SlabDesc> sl;
  fmm::bind_slabs(L, p->d_pack, p->d_scratch, es, sl);
  void* ds = nullptr;
  if ((st = dev_alloc(&ds, sizeof(fmm::SlabDesc) * sl.size())) != FMMFFT_OK) return st;
  p->d_slab = (fmm::SlabDesc*)ds;
  if (cudaMemcpy(ds, sl.data(), sizeof(fmm::SlabDesc) * sl.size(), cudaMemcpyHostToDevice) != cudaSuccess)
    return FMMFFT_ERR_CUDA;
  p->elements_plain = (int64_t)p->n[0] * p->n[1] * p->n[2] * p->n_dir;
  p->elements_compressed = L.elements;
  p->bytes_operator = (int64_t)(L.pack.size() * es + sizeof(fmm::SlabDesc) * sl.size() +
                                sizeof(fmm::GemmDesc) * flat.size());
  p->bytes_restore = (int64_t)(L.scratch * es);
  return FMMFFT_OK;
}

// Plan fields that describe a layout (ranks, restore shape), set before the
// support check so that it sees the layout's shared-memory needs.
void adopt_layout_shape(fmmfft_plan_s* p, const fmm::Layout& L) {
  p->yz_fmt = L.yz_fmt;
  p->rmax_a = L.rmax_a;
  p->rmax_b = L.rmax_b;
  for (int i = 0; i < 6; ++i) p->rmax[i] = L.rank[i];
  for (int i = 0; i < 3; ++i) p->mean_rank[i] = L.mean_rank[i];
  p->ranks3 = L.ranks3;
}

fmm::OperatorSpec spec_of(const fmmfft_plan_s* p) {
  fmm::OperatorSpec s;
  for (int i = 0; i < 3; ++i) {
    s.K[i] = p->K[i];
    s.n[i] = p->n[i];
  }
  s.L = p->L;
  s.a = p->a;
  s.k0 = p->k0;
  s.eps_re = p->eps_re;
  s.eps_im = p->eps_im;
  s.near_rule = p->near_rule;
  s.kappa = p->kappa;
  s.prefactor = p->prefactor;
  return s;
}

bool precision_supported(const fmmfft_plan_s* p) {
  return p->precision == FMMFFT_PREC_C128 || p->precision == FMMFFT_PREC_C64 ||
         p->precision == FMMFFT_PREC_C64_3XTF32 || p->precision == FMMFFT_PREC_C64_BF16X3 ||
         p->precision == FMMFFT_PREC_C64_TF32;
}

bool check_supported(fmmfft_plan_s* p) {
  fmm::TranslateArgs a = base_args(p);
  return fmm::translate_supported(a);
}

bool format_known(const fmmfft_plan_s* p) {
  if (p->format == FMMFFT_FORMAT_NONE) return true;
  if (p->format == FMMFFT_FORMAT_3D) return p->decomp == FMMFFT_DECOMP_TUCKER || p->decomp == FMMFFT_DECOMP_TT;
  return p->decomp == FMMFFT_DECOMP_TUCKER || p->decomp == FMMFFT_DECOMP_TT || p->decomp == FMMFFT_DECOMP_HTUCKER;
}

// FP64 host set-up of a compressed plan: operators (Eq. 7, Sec. II.B) and
// their decomposition in the plan's format (Algs. 1-3), as a layout.
void build_layout(const fmmfft_plan_s* p, fmm::Layout& L) {
  const fmm::OperatorSpec s = spec_of(p);
  const int nd = p->n_dir;
  if (p->format == FMMFFT_FORMAT_3D && p->decomp == FMMFFT_DECOMP_TUCKER) {
    std::vector<fmm::Tucker3> tk(nd);
    fmm::parallel_for(nd, [&](int d) {
      std::vector<cdouble> T;
      fmm::fft_operator(s, &p->khat[3 * d], T);
      fmm::hosvd3(T, p->n, p->tol, p->trunc_rule, tk[d]);
    });
    fmm::layout_tucker3d(tk, p->n, L);
    return;
  }
  if (p->format == FMMFFT_FORMAT_3D) {
    std::vector<fmm::TT3> tt(nd);
    fmm::parallel_for(nd, [&](int d) {
      std::vector<cdouble> T;
      fmm::fft_operator(s, &p->khat[3 * d], T);
      fmm::ttsvd3(T, p->n, p->tol, p->trunc_rule, tt[d]);
    });
    fmm::layout_tt3d(tt, p->n, L);
    return;
  }
  // 4D formats decompose T_4D over the whole direction grid (Sec. II.B: the
  // directions are the fourth mode).  A shard plan keeps the shared cores and
  // only its block's rows of the direction factor (U4, or U3 of TT), so every
  // shard restores its directions from one global decomposition, exactly as
  // the whole plan does.
  const bool shard = nd != p->n_dir_grid;
  std::vector<double> kh_all = p->khat, w_all;
  if (shard) fmm::direction_grid(p->L, p->nphi_rule == 0 ? 2 * (p->L + 1) : 2 * p->L + 1, kh_all, w_all);
  const int nd_all = shard ? p->n_dir_grid : nd;
  std::vector<std::vector<cdouble>> Tp(nd_all);
  fmm::parallel_for(nd_all, [&](int d) { fmm::fft_operator(s, &kh_all[3 * d], Tp[d]); });
  // rows dir_first .. dir_first + nd - 1 of a direction factor with r columns
  auto rows_of_block = [&](std::vector<cdouble>& U, int r) {
    if (!shard) return;
    std::vector<cdouble> sub(U.begin() + (size_t)p->dir_first * r, U.begin() + (size_t)(p->dir_first + nd) * r);
    U.swap(sub);
  };
  if (p->decomp == FMMFFT_DECOMP_TUCKER) {
    double n2 = 0.0;
    for (auto& T : Tp)
      for (auto& z : T) n2 += std::norm(z);
    fmm::Tucker4 tk;
    fmm::hosvd4(Tp, p->n, fmm::step_budget(std::sqrt(n2), p->tol, 4.0, p->trunc_rule), p->trunc_rule, tk);
    rows_of_block(tk.U[3], tk.r[3]);
    fmm::layout_tucker4d(tk, p->n, nd, L);
  } else if (p->decomp == FMMFFT_DECOMP_HTUCKER) {
    fmm::HTucker4 ht;
    fmm::htucker4(Tp, p->n, p->tol, p->trunc_rule, ht);
    rows_of_block(ht.U[3], ht.r[3]);
    fmm::layout_htucker(ht, p->n, nd, L);
  } else {
    fmm::TT4 tt;
    fmm::tt4_via_tucker(Tp, p->n, p->tol, p->trunc_rule, tt);
    rows_of_block(tt.U3, tt.r[2]);
    fmm::layout_tt4d(tt, p->n, nd, L);
  }
}

// FP64 relative error of a layout's restoration against the plan's own
// operator (Eq. 7, embedding and FFT), over all directions.
double measure_restore_error(const fmmfft_plan_s* p, const fmm::Layout& L) {
  const fmm::OperatorSpec s = spec_of(p);
  return fmm::restore_error_host(L, [&](int d, std::vector<cdouble>& T) { fmm::fft_operator(s, &p->khat[3 * d], T); });
}

// Adopt a compressed layout: support check, upload, common buffers.
int install_layout(fmmfft_plan_s* p, const fmm::Layout& L) {
  p->restore_err = -1.0;
  release_operator(p);
  p->layout = L;
  adopt_layout_shape(p, L);
  if (!check_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  int st = query_large_grid(p);
  if (st != FMMFFT_OK) return st;
  if ((st = upload_layout(p, L)) != FMMFFT_OK) return st;
  if ((st = ensure_slabs(p)) != FMMFFT_OK) return st;
  if ((st = ensure_common(p)) != FMMFFT_OK) return st;
  p->ready = true;
  if (p->measure_err) p->restore_err = measure_restore_error(p, L);
  return FMMFFT_OK;
}

const cdouble* as_cd(const double* x) { return reinterpret_cast<const cdouble*>(x); }

std::vector<cdouble> take(const cdouble*& src, size_t count) {
  std::vector<cdouble> v(src, src + count);
  src += count;
  return v;
}

}  // namespace

extern "C" {

const char* fmmfft_status_string(int s) {
  switch (s) {
    case FMMFFT_OK: return "ok";
    case FMMFFT_ERR_INVALID_ARG: return "invalid argument";
    case FMMFFT_ERR_NOT_COMPRESSED: return "plan has no operator yet (call fmmfft_compress or an import)";
    case FMMFFT_ERR_OOM: return "out of memory";
    case FMMFFT_ERR_CUDA: return "CUDA runtime error";
    case FMMFFT_ERR_UNSUPPORTED: return "sizes or format not supported by this build";
    case FMMFFT_ERR_DEVICE: return "a kernel reported a failure";
    case FMMFFT_ERR_IO: return "file input/output failed";
    case FMMFFT_ERR_TOO_LARGE:
      return "the translation needs more scratch than fmmfft_translate_noalloc's fixed 32 MiB buffer";
    default: return "unknown status";
  }
}

int fmmfft_plan_create(fmmfft_plan* out, int Nx, int Ny, int Nz, double a, double k0, int L,
                       int format, int decomp, double tol) {
  if (!out) return FMMFFT_ERR_INVALID_ARG;
  *out = nullptr;
  const int K[3] = {Nx, Ny, Nz};
  for (int i = 0; i < 3; ++i)
    if (K[i] < 2 || K[i] > 128) return FMMFFT_ERR_INVALID_ARG;
  if (!(a > 0) || !(k0 > 0) || !std::isfinite(a) || !std::isfinite(k0)) return FMMFFT_ERR_INVALID_ARG;
  if (L < 0 || L > 64) return FMMFFT_ERR_INVALID_ARG;
  if (format != FMMFFT_FORMAT_NONE && format != FMMFFT_FORMAT_3D && format != FMMFFT_FORMAT_4D)
    return FMMFFT_ERR_INVALID_ARG;
  if (decomp < FMMFFT_DECOMP_NONE || decomp > FMMFFT_DECOMP_HTUCKER) return FMMFFT_ERR_INVALID_ARG;
  if ((format == FMMFFT_FORMAT_NONE) != (decomp == FMMFFT_DECOMP_NONE)) return FMMFFT_ERR_INVALID_ARG;
  if (decomp == FMMFFT_DECOMP_HTUCKER && format != FMMFFT_FORMAT_4D) return FMMFFT_ERR_INVALID_ARG;
  if (decomp != FMMFFT_DECOMP_NONE && !(tol > 0 && tol < 1)) return FMMFFT_ERR_INVALID_ARG;
  fmmfft_plan_s* p = new (std::nothrow) fmmfft_plan_s();
  if (!p) return FMMFFT_ERR_OOM;
  for (int i = 0; i < 3; ++i) {
    p->K[i] = K[i];
    p->n[i] = embed_extent(K[i]);
  }
  p->a = a;
  p->k0 = k0;
  p->L = L;
  p->format = format;
  p->decomp = decomp;
  p->tol = tol;
  set_directions(p, 0, 0, 0);
  *out = p;
  return FMMFFT_OK;
}

int fmmfft_plan_set(fmmfft_plan p, int key, double v) {
  if (!p || (p->ready && key != FMMFFT_KEY_PROFILE && key != FMMFFT_KEY_HOST_BLOCKS)) return FMMFFT_ERR_INVALID_ARG;
  const int iv = (int)v;
  switch (key) {
    case FMMFFT_KEY_PRECISION:
      if (iv < FMMFFT_PREC_C128 || iv > FMMFFT_PREC_C64_TF32 || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->precision = iv;
      return FMMFFT_OK;
    case FMMFFT_KEY_NPHI_RULE:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      free_dev(p->d_weights);
      // a shard block that no longer fits the new grid falls back to the whole grid
      if (set_directions(p, iv, p->dir_first, p->dir_count) != FMMFFT_OK) set_directions(p, iv, 0, 0);
      return FMMFFT_OK;
    case FMMFFT_KEY_DIR_FIRST:
      if (iv != v) return FMMFFT_ERR_INVALID_ARG;
      free_dev(p->d_weights);
      return set_directions(p, p->nphi_rule, iv, p->dir_count);
    case FMMFFT_KEY_DIR_COUNT:
      if (iv != v) return FMMFFT_ERR_INVALID_ARG;
      free_dev(p->d_weights);
      return set_directions(p, p->nphi_rule, p->dir_first, iv);
    case FMMFFT_KEY_NEAR_RULE:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->near_rule = iv;
      return FMMFFT_OK;
    case FMMFFT_KEY_KAPPA:
      if (!(v >= 0) || !std::isfinite(v)) return FMMFFT_ERR_INVALID_ARG;
      p->kappa = v;
      return FMMFFT_OK;
    case FMMFFT_KEY_PREFACTOR:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->prefactor = iv;
      return FMMFFT_OK;
    case FMMFFT_KEY_TRUNC_RULE:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->trunc_rule = iv;
      return FMMFFT_OK;
    case FMMFFT_KEY_PROFILE:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->profile = iv == 1;
      return FMMFFT_OK;
    case FMMFFT_KEY_HOST_BLOCKS:
      if (iv < 0 || iv > kHostBlocksMax || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->host_blocks = iv;
      return FMMFFT_OK;
    case FMMFFT_KEY_EPS_R_RE:
      if (!(v > 0) || !std::isfinite(v)) return FMMFFT_ERR_INVALID_ARG;
      p->eps_re = v;
      return FMMFFT_OK;
    case FMMFFT_KEY_EPS_R_IM:
      if (!(v <= 0) || !std::isfinite(v)) return FMMFFT_ERR_INVALID_ARG;
      p->eps_im = v;
      return FMMFFT_OK;
    case FMMFFT_KEY_RESTORE_ERROR:
      if ((iv != 0 && iv != 1) || iv != v) return FMMFFT_ERR_INVALID_ARG;
      p->measure_err = iv == 1;
      return FMMFFT_OK;
    default:
      return FMMFFT_ERR_INVALID_ARG;
  }
}

int fmmfft_compress(fmmfft_plan p) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  if (!format_known(p) || !precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  int st;
  p->restore_err = -1.0;
  if (p->format == FMMFFT_FORMAT_NONE) {
    if (!check_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
    release_operator(p);
    if ((st = query_large_grid(p)) != FMMFFT_OK) return st;
    const fmm::OperatorSpec s = spec_of(p);
    std::vector<std::vector<cdouble>> ops(p->n_dir);
    fmm::parallel_for(p->n_dir, [&](int d) { fmm::fft_operator(s, &p->khat[3 * d], ops[d]); });
    st = upload_plain(p, [&](int d) { return ops[d].data(); });
    if (st != FMMFFT_OK) return st;
    if ((st = ensure_common(p)) != FMMFFT_OK) return st;
    p->ready = true;
    if (p->measure_err) p->restore_err = 0.0;   // stored as generated
  } else {
    fmm::Layout L;
    build_layout(p, L);
    if ((st = install_layout(p, L)) != FMMFFT_OK) return st;
  }
  p->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  return FMMFFT_OK;
}

int fmmfft_import_plain(fmmfft_plan p, const double* That) {
  if (!p || !That || p->format != FMMFFT_FORMAT_NONE) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  if (!check_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  p->restore_err = -1.0;
  release_operator(p);
  int st = query_large_grid(p);
  if (st != FMMFFT_OK) return st;
  const size_t per = (size_t)p->n[0] * p->n[1] * p->n[2];
  const cdouble* T = reinterpret_cast<const cdouble*>(That);
  st = upload_plain(p, [&](int d) { return T + per * d; });
  if (st != FMMFFT_OK) return st;
  if ((st = ensure_common(p)) != FMMFFT_OK) return st;
  p->ready = true;
  return FMMFFT_OK;
}

int fmmfft_import_tucker3d(fmmfft_plan p, const int* ranks, const double* core, const double* U1,
                           const double* U2, const double* U3) {
  if (!p || !ranks || !core || !U1 || !U2 || !U3) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_3D || p->decomp != FMMFFT_DECOMP_TUCKER) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  std::vector<fmm::Tucker3> tk(p->n_dir);
  const cdouble* c = as_cd(core);
  const cdouble* u[3] = {as_cd(U1), as_cd(U2), as_cd(U3)};
  for (int d = 0; d < p->n_dir; ++d) {
    for (int i = 0; i < 3; ++i) {
      const int r = ranks[3 * d + i];
      if (r < 1 || r > p->n[i]) return FMMFFT_ERR_INVALID_ARG;
      tk[d].r[i] = r;
    }
    tk[d].core = take(c, (size_t)tk[d].r[0] * tk[d].r[1] * tk[d].r[2]);
    for (int i = 0; i < 3; ++i) tk[d].U[i] = take(u[i], (size_t)p->n[i] * tk[d].r[i]);
  }
  fmm::Layout L;
  fmm::layout_tucker3d(tk, p->n, L);
  return install_layout(p, L);
}

int fmmfft_import_tt3d(fmmfft_plan p, const int* ranks, const double* U1, const double* C1, const double* U3) {
  if (!p || !ranks || !U1 || !C1 || !U3) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_3D || p->decomp != FMMFFT_DECOMP_TT) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  std::vector<fmm::TT3> tt(p->n_dir);
  const cdouble* u1 = as_cd(U1);
  const cdouble* c1 = as_cd(C1);
  const cdouble* u3 = as_cd(U3);
  const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
  for (int d = 0; d < p->n_dir; ++d) {
    const int r1 = ranks[2 * d], r2 = ranks[2 * d + 1];
    if (r1 < 1 || r1 > n1 || r2 < 1 || r2 > (int64_t)r1 * n2) return FMMFFT_ERR_INVALID_ARG;
    tt[d].r1 = r1;
    tt[d].r2 = r2;
    tt[d].U1 = take(u1, (size_t)n1 * r1);
    tt[d].C1 = take(c1, (size_t)r1 * n2 * r2);
    tt[d].U3 = take(u3, (size_t)n3 * r2);
  }
  fmm::Layout L;
  fmm::layout_tt3d(tt, p->n, L);
  return install_layout(p, L);
}

int fmmfft_import_tucker4d(fmmfft_plan p, const int* ranks, const double* core, const double* U1,
                           const double* U2, const double* U3, const double* U4) {
  if (!p || !ranks || !core || !U1 || !U2 || !U3 || !U4) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_4D || p->decomp != FMMFFT_DECOMP_TUCKER) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  const int dims[4] = {p->n[0], p->n[1], p->n[2], p->n_dir};
  fmm::Tucker4 tk;
  size_t nc = 1;
  for (int i = 0; i < 4; ++i) {
    if (ranks[i] < 1 || ranks[i] > dims[i]) return FMMFFT_ERR_INVALID_ARG;
    tk.r[i] = ranks[i];
    nc *= (size_t)ranks[i];
  }
  const cdouble* c = as_cd(core);
  tk.core = take(c, nc);
  const double* U[4] = {U1, U2, U3, U4};
  for (int i = 0; i < 4; ++i) {
    const cdouble* u = as_cd(U[i]);
    tk.U[i] = take(u, (size_t)dims[i] * tk.r[i]);
  }
  fmm::Layout L;
  fmm::layout_tucker4d(tk, p->n, p->n_dir, L);
  return install_layout(p, L);
}

int fmmfft_import_htucker(fmmfft_plan p, const int* ranks, const double* U1, const double* U2,
                          const double* U3, const double* U4, const double* C12, const double* C34,
                          const double* B) {
  if (!p || !ranks || !U1 || !U2 || !U3 || !U4 || !C12 || !C34 || !B) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_4D || p->decomp != FMMFFT_DECOMP_HTUCKER) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  const int dims[4] = {p->n[0], p->n[1], p->n[2], p->n_dir};
  fmm::HTucker4 ht;
  for (int i = 0; i < 6; ++i) {
    if (ranks[i] < 1) return FMMFFT_ERR_INVALID_ARG;
    ht.r[i] = ranks[i];
  }
  for (int i = 0; i < 4; ++i)
    if (ranks[i] > dims[i]) return FMMFFT_ERR_INVALID_ARG;
  if (ranks[4] > ranks[0] * ranks[1] || ranks[5] > ranks[2] * ranks[3]) return FMMFFT_ERR_INVALID_ARG;
  const double* U[4] = {U1, U2, U3, U4};
  for (int i = 0; i < 4; ++i) {
    const cdouble* u = as_cd(U[i]);
    ht.U[i] = take(u, (size_t)dims[i] * ht.r[i]);
  }
  const cdouble* c12 = as_cd(C12);
  const cdouble* c34 = as_cd(C34);
  const cdouble* b = as_cd(B);
  ht.C12 = take(c12, (size_t)ht.r[0] * ht.r[1] * ht.r[4]);
  ht.C34 = take(c34, (size_t)ht.r[2] * ht.r[3] * ht.r[5]);
  ht.B = take(b, (size_t)ht.r[4] * ht.r[5]);
  fmm::Layout L;
  fmm::layout_htucker(ht, p->n, p->n_dir, L);
  return install_layout(p, L);
}

int fmmfft_import_tt4d(fmmfft_plan p, const int* ranks, const double* U1, const double* C1, const double* C2,
                       const double* U3) {
  if (!p || !ranks || !U1 || !C1 || !C2 || !U3) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_4D || p->decomp != FMMFFT_DECOMP_TT) return FMMFFT_ERR_INVALID_ARG;
  if (!precision_supported(p)) return FMMFFT_ERR_UNSUPPORTED;
  const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
  fmm::TT4 tt;
  for (int i = 0; i < 3; ++i) {
    if (ranks[i] < 1) return FMMFFT_ERR_INVALID_ARG;
    tt.r[i] = ranks[i];
  }
  if (tt.r[0] > n1 || tt.r[2] > p->n_dir) return FMMFFT_ERR_INVALID_ARG;
  const cdouble* u1 = as_cd(U1);
  const cdouble* c1 = as_cd(C1);
  const cdouble* c2 = as_cd(C2);
  const cdouble* u3 = as_cd(U3);
  tt.U1 = take(u1, (size_t)n1 * tt.r[0]);
  tt.C1 = take(c1, (size_t)tt.r[0] * n2 * tt.r[1]);
  tt.C2 = take(c2, (size_t)tt.r[1] * n3 * tt.r[2]);
  tt.U3 = take(u3, (size_t)p->n_dir * tt.r[2]);
  fmm::Layout L;
  fmm::layout_tt4d(tt, p->n, p->n_dir, L);
  return install_layout(p, L);
}

int fmmfft_compress_host(fmmfft_plan p, int* ranks, double* restored) {
  if (!p || !ranks || p->format == FMMFFT_FORMAT_NONE || !format_known(p)) return FMMFFT_ERR_INVALID_ARG;
  const auto t0 = std::chrono::steady_clock::now();
  fmm::Layout L;
  build_layout(p, L);
  if (!p->ready) {
    // statistics of this host compression (ranks, memory saving, set-up time)
    adopt_layout_shape(p, L);
    p->elements_plain = (int64_t)p->n[0] * p->n[1] * p->n[2] * p->n_dir;
    p->elements_compressed = L.elements;
    p->setup_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    p->restore_err = p->measure_err ? measure_restore_error(p, L) : -1.0;
  }
  if (p->format == FMMFFT_FORMAT_3D) {
    std::memcpy(ranks, L.ranks3.data(), sizeof(int) * L.ranks3.size());
  } else {
    for (int i = 0; i < 6; ++i) ranks[i] = L.rank[i];
  }
  if (restored) {
    std::vector<cdouble> T;
    fmm::restore_host(L, T);
    std::memcpy(restored, T.data(), T.size() * sizeof(cdouble));
  }
  return FMMFFT_OK;
}

int fmmfft_translate(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* stream) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  if (!S_in || !S_out || nrhs < 1 || nrhs > 4096) return FMMFFT_ERR_INVALID_ARG;
  const size_t es = elem_bytes(p);
  const size_t field = (size_t)p->K[0] * p->K[1] * p->K[2];
  const size_t bytes = (size_t)p->n_dir * 2 * nrhs * field * es;
  const char* i0 = (const char*)S_in;
  const char* o0 = (const char*)S_out;
  if (i0 < o0 + bytes && o0 < i0 + bytes) return FMMFFT_ERR_INVALID_ARG;
  if (((uintptr_t)S_in | (uintptr_t)S_out) % es) return FMMFFT_ERR_INVALID_ARG;
  const size_t inter = (size_t)p->n_dir * 2 * nrhs * p->n[0] * p->K[1] * p->K[2] * es;
  if (inter > p->inter_bytes) {
    if (p->d_inter) {
      cudaStreamSynchronize((cudaStream_t)stream);
      free_dev(p->d_inter);
    }
    p->inter_bytes = 0;
    int st = dev_alloc(&p->d_inter, inter);
    if (st != FMMFFT_OK) return st;
    p->inter_bytes = inter;
  }
  fmm::TranslateArgs a = base_args(p);
  a.nrhs = nrhs;
  a.s_in = S_in;
  a.s_out = S_out;
  a.inter = p->d_inter;
  a.stream = (cudaStream_t)stream;
  p->last_stream = a.stream;
  if (p->profile) {
    if (!p->events[0])
      for (auto& ev : p->events)
        if (cudaEventCreate(&ev) != cudaSuccess) return FMMFFT_ERR_CUDA;
    a.events = p->events;
    p->profiled_run = true;
  }
  cudaError_t e = fmm::launch_translate(a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

}  // extern "C"

namespace fmm {

int translate_scratch_bytes(fmmfft_plan p, int nrhs, size_t* bytes) {
  if (!p || !bytes) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  if (nrhs < 1 || nrhs > 4096) return FMMFFT_ERR_INVALID_ARG;
  *bytes = (size_t)p->n_dir * 2 * nrhs * p->n[0] * p->K[1] * p->K[2] * elem_bytes(p);
  return FMMFFT_OK;
}

int plan_intermediate(fmmfft_plan p, int nrhs, void* stream, void** inter, size_t* bytes) {
  size_t need = 0;
  int st = translate_scratch_bytes(p, nrhs, &need);
  if (st != FMMFFT_OK) return st;
  if (need > p->inter_bytes) {
    if (p->d_inter) {
      cudaStreamSynchronize((cudaStream_t)stream);
      free_dev(p->d_inter);
    }
    p->inter_bytes = 0;
    if ((st = dev_alloc(&p->d_inter, need)) != FMMFFT_OK) return st;
    p->inter_bytes = need;
  }
  *inter = p->d_inter;
  *bytes = p->inter_bytes;
  return FMMFFT_OK;
}

void plan_set_last_stream(fmmfft_plan p, void* stream) {
  if (p) p->last_stream = (cudaStream_t)stream;
}

int translate_args_for(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* scratch, size_t scratch_bytes,
                       TranslateArgs* out) {
  size_t need = 0;
  int st = translate_scratch_bytes(p, nrhs, &need);
  if (st != FMMFFT_OK) return st;
  if (!S_in || !S_out || !scratch || !out) return FMMFFT_ERR_INVALID_ARG;
  const size_t es = elem_bytes(p);
  const size_t bytes = (size_t)p->n_dir * 2 * nrhs * p->K[0] * p->K[1] * p->K[2] * es;
  const char* i0 = (const char*)S_in;
  const char* o0 = (const char*)S_out;
  if (i0 < o0 + bytes && o0 < i0 + bytes) return FMMFFT_ERR_INVALID_ARG;
  if (((uintptr_t)S_in | (uintptr_t)S_out | (uintptr_t)scratch) % es) return FMMFFT_ERR_INVALID_ARG;
  if (need > scratch_bytes) return FMMFFT_ERR_TOO_LARGE;
  fmm::TranslateArgs a = base_args(p);
  a.nrhs = nrhs;
  a.s_in = S_in;
  a.s_out = S_out;
  a.inter = scratch;
  a.events = nullptr;
  *out = a;
  return FMMFFT_OK;
}

int translate_into(fmmfft_plan p, const void* S_in, void* S_out, int nrhs, void* stream,
                   void* scratch, size_t scratch_bytes) {
  size_t need = 0;
  int st = translate_scratch_bytes(p, nrhs, &need);
  if (st != FMMFFT_OK) return st;
  if (!S_in || !S_out || !scratch) return FMMFFT_ERR_INVALID_ARG;
  const size_t es = elem_bytes(p);
  const size_t bytes = (size_t)p->n_dir * 2 * nrhs * p->K[0] * p->K[1] * p->K[2] * es;
  const char* i0 = (const char*)S_in;
  const char* o0 = (const char*)S_out;
  if (i0 < o0 + bytes && o0 < i0 + bytes) return FMMFFT_ERR_INVALID_ARG;
  if (((uintptr_t)S_in | (uintptr_t)S_out | (uintptr_t)scratch) % es) return FMMFFT_ERR_INVALID_ARG;
  if (need > scratch_bytes) return FMMFFT_ERR_TOO_LARGE;
  fmm::TranslateArgs a = base_args(p);
  a.nrhs = nrhs;
  a.s_in = S_in;
  a.s_out = S_out;
  a.inter = scratch;
  a.stream = (cudaStream_t)stream;
  a.events = nullptr;
  p->last_stream = a.stream;
  if (fmm::launch_translate(a) != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

}  // namespace fmm

extern "C" {

int fmmfft_translate_host(fmmfft_plan p, const void* S_in_host, void* S_out_host, int nrhs,
                          void* stream) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  if (!S_in_host || !S_out_host || nrhs < 1 || nrhs > 4096) return FMMFFT_ERR_INVALID_ARG;
  const size_t per_dir = (size_t)2 * nrhs * p->K[0] * p->K[1] * p->K[2] * elem_bytes(p);
  const size_t bytes = (size_t)p->n_dir * per_dir;
  cudaStream_t s = (cudaStream_t)stream;
  if (2 * bytes > p->io_bytes) {
    if (p->d_io) {
      cudaStreamSynchronize(s);
      free_dev(p->d_io);
    }
    p->io_bytes = 0;
    int st = dev_alloc(&p->d_io, 2 * bytes);
    if (st != FMMFFT_OK) return st;
    p->io_bytes = 2 * bytes;
  }
  char* din = (char*)p->d_io;
  char* dout = din + bytes;
  const int want = p->host_blocks > 0 ? p->host_blocks : kHostBlocksDefault;
  const int blocks = p->profile ? 1 : std::min(want, p->n_dir);
  if (blocks <= 1) {
    if (cudaMemcpyAsync(din, S_in_host, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess) return FMMFFT_ERR_CUDA;
    int st = fmmfft_translate(p, din, dout, nrhs, stream);
    if (st != FMMFFT_OK) return st;
    if (cudaMemcpyAsync(S_out_host, dout, bytes, cudaMemcpyDeviceToHost, s) != cudaSuccess) return FMMFFT_ERR_CUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? FMMFFT_OK : FMMFFT_ERR_CUDA;
  }
  // Pipeline over blocks of directions: the copy-in of every block is queued
  // on one copy stream, the translation of block k waits for its copy-in, and
  // its copy-out runs on a second copy stream while block k + 1 translates.
  void* inter = nullptr;
  size_t ib = 0;
  int st = fmm::plan_intermediate(p, nrhs, stream, &inter, &ib);
  if (st != FMMFFT_OK) return st;
  if (!p->h2d) {
    if (cudaStreamCreateWithFlags(&p->h2d, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithFlags(&p->d2h, cudaStreamNonBlocking) != cudaSuccess)
      return FMMFFT_ERR_CUDA;
    for (auto& ev : p->hev)
      if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return FMMFFT_ERR_CUDA;
  }
  cudaEvent_t ev_start = p->hev[0], ev_done = p->hev[1];
  cudaEvent_t* ev_in = p->hev + 2;
  cudaEvent_t* ev_out = ev_in + kHostBlocksMax;
  // on a failure part-way, let the copies already queued finish before
  // returning: they read and write the caller's host buffers
  auto fail = [&]() {
    cudaGetLastError();
    cudaStreamSynchronize(p->h2d);
    cudaStreamSynchronize(p->d2h);
    cudaStreamSynchronize(s);
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  };
  const int per = (p->n_dir + blocks - 1) / blocks;
  const char* hin = (const char*)S_in_host;
  char* hout = (char*)S_out_host;
  // the copies must follow earlier work of `stream` on these buffers
  if (cudaEventRecord(ev_start, s) != cudaSuccess || cudaStreamWaitEvent(p->h2d, ev_start, 0) != cudaSuccess ||
      cudaStreamWaitEvent(p->d2h, ev_start, 0) != cudaSuccess)
    return fail();
  for (int k = 0, p0 = 0; p0 < p->n_dir; ++k, p0 += per) {
    const size_t off = (size_t)p0 * per_dir, len = (size_t)std::min(per, p->n_dir - p0) * per_dir;
    if (cudaMemcpyAsync(din + off, hin + off, len, cudaMemcpyHostToDevice, p->h2d) != cudaSuccess ||
        cudaEventRecord(ev_in[k], p->h2d) != cudaSuccess)
      return fail();
  }
  p->last_stream = s;
  for (int k = 0, p0 = 0; p0 < p->n_dir; ++k, p0 += per) {
    const int nw = std::min(per, p->n_dir - p0);
    const size_t off = (size_t)p0 * per_dir, len = (size_t)nw * per_dir;
    if (cudaStreamWaitEvent(s, ev_in[k], 0) != cudaSuccess) return fail();
    fmm::TranslateArgs a = base_args(p);
    a.nrhs = nrhs;
    a.s_in = din;
    a.s_out = dout;
    a.inter = inter;
    a.stream = s;
    a.p0 = p0;
    a.nw = nw;
    a.prepass = k == 0;
    if (fmm::launch_translate(a) != cudaSuccess) return fail();
    if (cudaEventRecord(ev_out[k], s) != cudaSuccess || cudaStreamWaitEvent(p->d2h, ev_out[k], 0) != cudaSuccess ||
        cudaMemcpyAsync(hout + off, dout + off, len, cudaMemcpyDeviceToHost, p->d2h) != cudaSuccess)
      return fail();
  }
  if (cudaEventRecord(ev_done, p->d2h) != cudaSuccess || cudaStreamWaitEvent(s, ev_done, 0) != cudaSuccess)
    return fail();
  return cudaStreamSynchronize(s) == cudaSuccess ? FMMFFT_OK : FMMFFT_ERR_CUDA;
}

int fmmfft_operator_host(fmmfft_plan p, int d, double* out) {
  if (!p || !out || d < 0 || d >= p->n_dir) return FMMFFT_ERR_INVALID_ARG;
  std::vector<cdouble> T;
  fmm::fft_operator(spec_of(p), &p->khat[3 * d], T);
  std::memcpy(out, T.data(), T.size() * sizeof(cdouble));
  return FMMFFT_OK;
}

int fmmfft_compress_direction_host(fmmfft_plan p, int d, int* ranks, double* restored) {
  if (!p || !ranks || d < 0 || d >= p->n_dir) return FMMFFT_ERR_INVALID_ARG;
  if (p->format != FMMFFT_FORMAT_3D || p->decomp != FMMFFT_DECOMP_TUCKER) return FMMFFT_ERR_INVALID_ARG;
  std::vector<cdouble> T;
  fmm::fft_operator(spec_of(p), &p->khat[3 * d], T);
  fmm::Tucker3 tk;
  fmm::hosvd3(T, p->n, p->tol, p->trunc_rule, tk);
  for (int i = 0; i < 3; ++i) ranks[i] = tk.r[i];
  if (restored) {
    const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
    const int r1 = tk.r[0], r2 = tk.r[1], r3 = tk.r[2];
    cdouble* o = reinterpret_cast<cdouble*>(restored);
    for (int x = 0; x < n1; ++x)
      for (int y = 0; y < n2; ++y)
        for (int z = 0; z < n3; ++z) {
          cdouble acc(0.0, 0.0);
          for (int a = 0; a < r1; ++a)
            for (int b = 0; b < r2; ++b) {
              const cdouble ab = tk.U[0][(size_t)x * r1 + a] * tk.U[1][(size_t)y * r2 + b];
              const cdouble* c = &tk.core[((size_t)a * r2 + b) * r3];
              cdouble s(0.0, 0.0);
              for (int k = 0; k < r3; ++k) s += c[k] * tk.U[2][(size_t)z * r3 + k];
              acc += ab * s;
            }
          o[((size_t)x * n2 + y) * n3 + z] = acc;
        }
  }
  return FMMFFT_OK;
}

int fmmfft_plan_stats(fmmfft_plan p, fmmfft_stats* o) {
  if (!p || !o) return FMMFFT_ERR_INVALID_ARG;
  std::memset(o, 0, sizeof(*o));
  o->n_dir = p->n_dir;
  o->L = p->L;
  for (int i = 0; i < 3; ++i) {
    o->K[i] = p->K[i];
    o->n[i] = p->n[i];
    o->mean_rank[i] = p->mean_rank[i];
  }
  o->format = p->format;
  o->decomp = p->decomp;
  o->precision = p->precision;
  for (int i = 0; i < 6; ++i) o->max_rank[i] = p->rmax[i];
  o->elements_plain = p->elements_plain;
  o->elements_compressed = p->elements_compressed;
  o->saving = p->elements_plain ? 1.0 - (double)p->elements_compressed / (double)p->elements_plain : 0.0;
  o->device_bytes_operator = p->bytes_operator;
  o->device_bytes_scratch = (int64_t)(p->inter_bytes + p->io_bytes + p->slabs_bytes) + p->bytes_restore;
  o->setup_seconds = p->setup_seconds;
  o->restore_rel_err = p->restore_err;
  if (p->ready) {
    const fmm::TranslateArgs a = base_args(p);
    o->restore_on_tensor_cores = a.tc == 1 && a.tc_single ? 3 : a.tc;
    o->kernel_launches = a.n_stages + 3;
    o->large_planes = a.large;
    o->schedule[0] = p->sched.xrows;
    o->schedule[1] = p->sched.tc_slab;
    o->schedule[2] = p->sched.tc_gemm;
    o->schedule[3] = p->sched.no_overlap;
  }
  return FMMFFT_OK;
}

namespace {

// Shared checks of the far-field entry points; fills the launch arguments.
int farfield_args(fmmfft_plan p, const void* P, const void* in, void* out, int nb, int nrhs, void* stream,
                  size_t in_elems_per_box, size_t out_elems_per_box, fmm::FarFieldArgs& a) {
  if (!p || !P || !in || !out || nb < 1 || nrhs < 1 || nrhs > 4096) return FMMFFT_ERR_INVALID_ARG;
  if (nb > fmm::kFarFieldMaxNb) return FMMFFT_ERR_UNSUPPORTED;
  const bool fp64 = p->precision == FMMFFT_PREC_C128;
  const size_t es = fp64 ? 16 : 8;
  const size_t V = (size_t)p->K[0] * p->K[1] * p->K[2];
  if (((uintptr_t)P | (uintptr_t)in | (uintptr_t)out) % es) return FMMFFT_ERR_INVALID_ARG;
  const char* o0 = (const char*)out;
  const size_t ob = out_elems_per_box * V * es;
  const void* srcs[2] = {P, in};
  const size_t sb[2] = {(size_t)p->n_dir * 2 * nb * V * es, in_elems_per_box * V * es};
  for (int k = 0; k < 2; ++k) {
    const char* s0 = (const char*)srcs[k];
    if (s0 < o0 + ob && o0 < s0 + sb[k]) return FMMFFT_ERR_INVALID_ARG;   // output aliases an input
  }
  if (!p->d_weights) {
    void* w = nullptr;
    int st = dev_alloc(&w, sizeof(double) * (size_t)std::max(p->n_dir, 1));
    if (st != FMMFFT_OK) return st;
    if (cudaMemcpy(w, p->weights.data(), sizeof(double) * p->n_dir, cudaMemcpyHostToDevice) != cudaSuccess) {
      free_dev(w);
      cudaGetLastError();
      return FMMFFT_ERR_CUDA;
    }
    p->d_weights = w;
  }
  a.P = P;
  a.in = in;
  a.out = out;
  a.w = (const double*)p->d_weights;
  a.V = (int64_t)V;
  a.nb = nb;
  a.nrhs = nrhs;
  a.n_dir = p->n_dir;
  a.fp64 = fp64;
  a.stream = (cudaStream_t)stream;
  return FMMFFT_OK;
}

}  // namespace

int fmmfft_aggregate(fmmfft_plan p, const void* patterns, const void* currents, void* A, int nb, int nrhs,
                     void* stream) {
  fmm::FarFieldArgs a;
  int st = farfield_args(p, patterns, currents, A, nb, nrhs, stream, (size_t)nb * (nrhs > 0 ? nrhs : 0),
                         (size_t)(p ? p->n_dir : 0) * 2 * (nrhs > 0 ? nrhs : 0), a);
  if (st != FMMFFT_OK) return st;
  cudaError_t e = fmm::launch_aggregate(a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

int fmmfft_disaggregate(fmmfft_plan p, const void* patterns, const void* B, void* y, int nb, int nrhs,
                        void* stream) {
  fmm::FarFieldArgs a;
  int st = farfield_args(p, patterns, B, y, nb, nrhs, stream, (size_t)(p ? p->n_dir : 0) * 2 * (nrhs > 0 ? nrhs : 0),
                         (size_t)nb * (nrhs > 0 ? nrhs : 0), a);
  if (st != FMMFFT_OK) return st;
  cudaError_t e = fmm::launch_disaggregate(a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

int fmmfft_translate_disaggregate(fmmfft_plan p, const void* S_in, const void* patterns, void* y, int nb, int nrhs,
                                  void* stream) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  fmm::FarFieldArgs fa;
  // the fields S_in play the role of the far-field input for the aliasing
  // and alignment checks: y must overlap neither them nor the patterns
  int st = farfield_args(p, patterns, S_in, y, nb, nrhs, stream, (size_t)p->n_dir * 2 * (nrhs > 0 ? nrhs : 0),
                         (size_t)nb * (nrhs > 0 ? nrhs : 0), fa);
  if (st != FMMFFT_OK) return st;
  if (p->K[0] > 128) return FMMFFT_ERR_UNSUPPORTED;
  void* inter = nullptr;
  size_t ib = 0;
  if ((st = fmm::plan_intermediate(p, nrhs, stream, &inter, &ib)) != FMMFFT_OK) return st;
  fmm::XDisArgs d;
  d.P = patterns;
  d.w = fa.w;
  d.y = y;
  d.nb = nb;
  fmm::TranslateArgs a = base_args(p);
  a.nrhs = nrhs;
  a.s_in = S_in;
  a.s_out = nullptr;
  a.inter = inter;
  a.stream = (cudaStream_t)stream;
  a.dis = &d;
  p->last_stream = a.stream;
  if (p->profile) {
    if (!p->events[0])
      for (auto& ev : p->events)
        if (cudaEventCreate(&ev) != cudaSuccess) return FMMFFT_ERR_CUDA;
    a.events = p->events;
    p->profiled_run = true;
  }
  cudaError_t e = fmm::launch_translate(a);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  return FMMFFT_OK;
}

int fmmfft_plan_set_occupancy(fmmfft_plan p, const unsigned char* occupied) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  const size_t V = (size_t)p->K[0] * p->K[1] * p->K[2];
  const size_t rows = (size_t)p->K[1] * p->K[2];
  // box mask, then per x-line: whether any box of the line is occupied; a
  // cleared mask is stored as a full one so that a launch captured earlier
  // keeps valid memory
  std::vector<unsigned char> h(V + rows, 1);
  if (occupied) {
    for (size_t r = 0; r < rows; ++r) {
      unsigned char any = 0;
      for (int x = 0; x < p->K[0]; ++x) {
        const unsigned char o = occupied[r * p->K[0] + x] ? 1 : 0;
        h[r * p->K[0] + x] = o;
        any |= o;
      }
      h[V + r] = any;
    }
  }
  // the plan's work in flight may read the previous mask
  if (p->d_occ && cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  if (!p->d_occ) {
    if (!occupied) return FMMFFT_OK;
    int st = dev_alloc(&p->d_occ, V + rows);
    if (st != FMMFFT_OK) return st;
  }
  if (cudaMemcpy(p->d_occ, h.data(), V + rows, cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaGetLastError();
    return FMMFFT_ERR_CUDA;
  }
  p->occ_set = occupied != nullptr;
  return FMMFFT_OK;
}

int fmmfft_multipole_count(double a, double k0, double eps_re, double eps_im, double digits, int* L_out) {
  if (!L_out || !(a > 0) || !(k0 > 0) || !(eps_re > 0) || !(eps_im <= 0) || !(digits > 0) ||
      !std::isfinite(a * k0 * eps_re * eps_im * digits))
    return FMMFFT_ERR_INVALID_ARG;
  *L_out = fmm::multipole_count(a, k0, eps_re, eps_im, digits);
  return FMMFFT_OK;
}

int fmmfft_plan_ranks(fmmfft_plan p, int* ranks) {
  if (!p || !ranks || !p->ready || p->format != FMMFFT_FORMAT_3D) return FMMFFT_ERR_INVALID_ARG;
  std::memcpy(ranks, p->ranks3.data(), sizeof(int) * p->ranks3.size());
  return FMMFFT_OK;
}

int fmmfft_plan_directions(fmmfft_plan p, double* khat, double* weights) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (khat) std::memcpy(khat, p->khat.data(), sizeof(double) * 3 * p->n_dir);
  if (weights) std::memcpy(weights, p->weights.data(), sizeof(double) * p->n_dir);
  return FMMFFT_OK;
}

int fmmfft_stage_times(fmmfft_plan p, float* ms) {
  if (!p || !ms || !p->profiled_run) return FMMFFT_ERR_INVALID_ARG;
  if (cudaEventSynchronize(p->events[FMMFFT_NUM_STAGES]) != cudaSuccess) return FMMFFT_ERR_CUDA;
  for (int i = 0; i < FMMFFT_NUM_STAGES; ++i)
    if (cudaEventElapsedTime(&ms[i], p->events[i], p->events[i + 1]) != cudaSuccess) return FMMFFT_ERR_CUDA;
  return FMMFFT_OK;
}

int fmmfft_poll_status(fmmfft_plan p, int* device_status) {
  if (!p || !device_status) return FMMFFT_ERR_INVALID_ARG;
  *device_status = 0;
  if (!p->d_status) return FMMFFT_OK;
  if (cudaStreamSynchronize(p->last_stream) != cudaSuccess) return FMMFFT_ERR_CUDA;
  if (cudaMemcpy(device_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return FMMFFT_ERR_CUDA;
  if (cudaMemset(p->d_status, 0, sizeof(int)) != cudaSuccess) return FMMFFT_ERR_CUDA;
  return FMMFFT_OK;
}

// ---------------------------------------------------------------------------
// plan files: header, options, and for compressed plans the stored factors
// with their restore schedule (the FP64 set-up is not repeated on load)
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

const char kMagic[8] = {'F', 'M', 'M', 'F', 'F', 'T', 'P', '1'};
const uint32_t kFileVersion = 3;   // 2: medium permittivity after trunc_rule; 3: direction block

struct Writer {
  FILE* f;
  bool ok = true;
  template <typename T> void put(const T& v) { ok = ok && fwrite(&v, sizeof(T), 1, f) == 1; }
  template <typename T> void put_vec(const std::vector<T>& v) {
    put<uint64_t>(v.size());
    if (!v.empty()) ok = ok && fwrite(v.data(), sizeof(T), v.size(), f) == v.size();
  }
  void put_ref(const fmm::BufRef& r) { put<int32_t>(r.buf); put<int64_t>(r.off); }
};

struct Reader {
  FILE* f;
  bool ok = true;
  template <typename T> T get() {
    T v{};
    ok = ok && fread(&v, sizeof(T), 1, f) == 1;
    return v;
  }
  template <typename T> void get_vec(std::vector<T>& v, uint64_t limit) {
    const uint64_t n = get<uint64_t>();
    if (!ok || n > limit) { ok = false; return; }
    v.resize(n);
    if (n) ok = ok && fread(v.data(), sizeof(T), n, f) == n;
  }
  fmm::BufRef get_ref() {
    fmm::BufRef r;
    r.buf = get<int32_t>();
    r.off = get<int64_t>();
    if (r.buf != 0 && r.buf != 1) ok = false;
    return r;
  }
};

}  // namespace

extern "C" {

int fmmfft_plan_save(fmmfft_plan p, const char* path) {
  if (!p || !path) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  FILE* f = std::fopen(path, "wb");
  if (!f) return FMMFFT_ERR_IO;
  Writer w{f};
  if (fwrite(kMagic, 1, 8, f) != 8) w.ok = false;
  w.put<uint32_t>(kFileVersion);
  for (int i = 0; i < 3; ++i) w.put<int32_t>(p->K[i]);
  w.put<int32_t>(p->L);
  w.put<double>(p->a);
  w.put<double>(p->k0);
  w.put<double>(p->tol);
  w.put<int32_t>(p->format);
  w.put<int32_t>(p->decomp);
  w.put<int32_t>(p->precision);
  w.put<int32_t>(p->nphi_rule);
  w.put<int32_t>(p->near_rule);
  w.put<double>(p->kappa);
  w.put<int32_t>(p->prefactor);
  w.put<int32_t>(p->trunc_rule);
  w.put<double>(p->eps_re);
  w.put<double>(p->eps_im);
  w.put<int32_t>(p->dir_first);
  w.put<int32_t>(p->dir_count);
  w.put<int32_t>(p->n_dir);
  if (p->format != FMMFFT_FORMAT_NONE) {
    const fmm::Layout& L = p->layout;
    for (int i = 0; i < 3; ++i) w.put<int32_t>(L.n[i]);
    w.put<int32_t>(L.n_dir);
    w.put<int32_t>(L.yz_fmt);
    w.put_vec(L.pack);
    w.put<int64_t>(L.scratch);
    w.put<uint64_t>(L.stages.size());
    for (const auto& st : L.stages) {
      w.put<uint64_t>(st.size());
      for (const auto& g : st) {
        w.put_ref(g.A);
        w.put_ref(g.B);
        w.put_ref(g.C);
        w.put<int32_t>(g.M);
        w.put<int32_t>(g.N);
        w.put<int32_t>(g.K);
      }
    }
    w.put<uint64_t>(L.slabs.size());
    for (const auto& sl : L.slabs) {
      w.put_ref(sl.h);
      w.put_ref(sl.u2);
      w.put_ref(sl.u3);
      w.put<int64_t>(sl.hx);
      w.put<int32_t>(sl.ra);
      w.put<int32_t>(sl.rb);
    }
    w.put<int64_t>(L.elements);
    for (int i = 0; i < 6; ++i) w.put<int32_t>(L.rank[i]);
    for (int i = 0; i < 3; ++i) w.put<double>(L.mean_rank[i]);
    w.put_vec(L.ranks3);
  }
  const bool closed = std::fclose(f) == 0;
  return (w.ok && closed) ? FMMFFT_OK : FMMFFT_ERR_IO;
}

int fmmfft_plan_load(fmmfft_plan* out, const char* path) {
  if (!out || !path) return FMMFFT_ERR_INVALID_ARG;
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) return FMMFFT_ERR_IO;
  Reader r{f};
  char magic[8] = {};
  const bool got = fread(magic, 1, 8, f) == 8;
  if (!got || std::memcmp(magic, kMagic, 8) != 0 || r.get<uint32_t>() != kFileVersion) {
    std::fclose(f);
    return got ? FMMFFT_ERR_INVALID_ARG : FMMFFT_ERR_IO;
  }
  int K[3];
  for (int i = 0; i < 3; ++i) K[i] = r.get<int32_t>();
  const int L = r.get<int32_t>();
  const double a = r.get<double>(), k0 = r.get<double>(), tol = r.get<double>();
  const int format = r.get<int32_t>(), decomp = r.get<int32_t>(), precision = r.get<int32_t>();
  const int nphi_rule = r.get<int32_t>(), near_rule = r.get<int32_t>();
  const double kappa = r.get<double>();
  const int prefactor = r.get<int32_t>(), trunc_rule = r.get<int32_t>();
  const double eps_re = r.get<double>(), eps_im = r.get<double>();
  const int dir_first = r.get<int32_t>(), dir_count = r.get<int32_t>();
  const int n_dir = r.get<int32_t>();
  fmmfft_plan p = nullptr;
  int st = r.ok ? fmmfft_plan_create(&p, K[0], K[1], K[2], a, k0, L, format, decomp, tol) : FMMFFT_ERR_IO;
  const std::pair<int, double> opts[] = {{FMMFFT_KEY_PRECISION, precision}, {FMMFFT_KEY_NPHI_RULE, nphi_rule},
                                         {FMMFFT_KEY_NEAR_RULE, near_rule},  {FMMFFT_KEY_KAPPA, kappa},
                                         {FMMFFT_KEY_PREFACTOR, prefactor},  {FMMFFT_KEY_TRUNC_RULE, trunc_rule},
                                         {FMMFFT_KEY_EPS_R_RE, eps_re},      {FMMFFT_KEY_EPS_R_IM, eps_im},
                                         {FMMFFT_KEY_DIR_COUNT, dir_count},  {FMMFFT_KEY_DIR_FIRST, dir_first}};
  for (const auto& o : opts)
    if (st == FMMFFT_OK) st = fmmfft_plan_set(p, o.first, o.second);
  if (st == FMMFFT_OK && p->n_dir != n_dir) st = FMMFFT_ERR_INVALID_ARG;
  if (st == FMMFFT_OK && format == FMMFFT_FORMAT_NONE) {
    std::fclose(f);
    f = nullptr;
    st = fmmfft_compress(p);
  } else if (st == FMMFFT_OK) {
    fmm::Layout Lt;
    const uint64_t big = (uint64_t)1 << 40;
    for (int i = 0; i < 3; ++i) Lt.n[i] = r.get<int32_t>();
    Lt.n_dir = r.get<int32_t>();
    Lt.yz_fmt = r.get<int32_t>();
    r.get_vec(Lt.pack, big);
    Lt.scratch = r.get<int64_t>();
    const uint64_t nst = r.get<uint64_t>();
    if (nst > (uint64_t)fmm::kMaxGemmStages) r.ok = false;
    for (uint64_t s = 0; r.ok && s < nst; ++s) {
      const uint64_t cnt = r.get<uint64_t>();
      if (cnt > (uint64_t)1 << 24) { r.ok = false; break; }
      std::vector<fmm::GemmSpec> stage(cnt);
      for (auto& g : stage) {
        g.A = r.get_ref();
        g.B = r.get_ref();
        g.C = r.get_ref();
        g.M = r.get<int32_t>();
        g.N = r.get<int32_t>();
        g.K = r.get<int32_t>();
      }
      Lt.stages.push_back(stage);
    }
    const uint64_t ns = r.get<uint64_t>();
    if (ns != (uint64_t)n_dir) r.ok = false;
    for (uint64_t s = 0; r.ok && s < ns; ++s) {
      fmm::SlabSpec sl;
      sl.h = r.get_ref();
      sl.u2 = r.get_ref();
      sl.u3 = r.get_ref();
      sl.hx = r.get<int64_t>();
      sl.ra = r.get<int32_t>();
      sl.rb = r.get<int32_t>();
      Lt.slabs.push_back(sl);
    }
    Lt.elements = r.get<int64_t>();
    for (int i = 0; i < 6; ++i) Lt.rank[i] = r.get<int32_t>();
    for (int i = 0; i < 3; ++i) Lt.mean_rank[i] = r.get<double>();
    r.get_vec(Lt.ranks3, (uint64_t)n_dir * 3);
    Lt.rmax_a = 0;
    Lt.rmax_b = 0;
    for (const auto& sl : Lt.slabs) {
      Lt.rmax_a = std::max(Lt.rmax_a, sl.ra);
      Lt.rmax_b = std::max(Lt.rmax_b, sl.rb);
    }
    // every reference must stay inside the buffers it names
    const int64_t sizes[2] = {(int64_t)Lt.pack.size(), Lt.scratch};
    auto inside = [&](const fmm::BufRef& b, int64_t count) {
      return b.off >= 0 && count >= 0 && b.off + count <= sizes[b.buf];
    };
    for (const auto& stage : Lt.stages)
      for (const auto& g : stage)
        if (g.M < 1 || g.N < 1 || g.K < 1 || !inside(g.A, (int64_t)g.M * g.K) ||
            !inside(g.B, (int64_t)g.K * g.N) || !inside(g.C, (int64_t)g.M * g.N) || g.C.buf != 1)
          r.ok = false;
    for (const auto& sl : Lt.slabs)
      if (sl.rb < 1 || sl.ra < 0 ||
          !inside(sl.h, sl.hx * (int64_t)(Lt.n[0] - 1) + (int64_t)(Lt.yz_fmt == 1 ? sl.ra : Lt.n[1]) * sl.rb) ||
          (sl.ra > 0 && !inside(sl.u2, (int64_t)Lt.n[1] * sl.ra)) || !inside(sl.u3, (int64_t)Lt.n[2] * sl.rb))
        r.ok = false;
    for (int i = 0; i < 3; ++i)
      if (Lt.n[i] != p->n[i]) r.ok = false;
    if (Lt.n_dir != n_dir || (Lt.yz_fmt != 1 && Lt.yz_fmt != 2)) r.ok = false;
    std::fclose(f);
    f = nullptr;
    st = r.ok ? install_layout(p, Lt) : FMMFFT_ERR_INVALID_ARG;
  }
  if (f) std::fclose(f);
  if (st != FMMFFT_OK) {
    if (p) fmmfft_plan_destroy(p);
    return st;
  }
  *out = p;
  return FMMFFT_OK;
}

// ---------------------------------------------------------------------------
// autotuner: time the plan's candidate schedules, keep the fastest
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

std::string tune_signature(const fmmfft_plan_s* p, int nrhs) {
  int dev = 0;
  cudaDeviceProp prop;
  std::string name = "unknown";
  int sms = 0;
  if (cudaGetDevice(&dev) == cudaSuccess && cudaGetDeviceProperties(&prop, dev) == cudaSuccess) {
    name = prop.name;
    sms = prop.multiProcessorCount;
  }
  cudaGetLastError();
  for (auto& c : name)
    if (c == ' ' || c == ';') c = '_';
  std::ostringstream o;
  o << "dev=" << name << ";sm=" << sms << ";K=" << p->K[0] << "," << p->K[1] << "," << p->K[2]
    << ";n_dir=" << p->n_dir << ";fmt=" << p->format << ";dec=" << p->decomp << ";prec=" << p->precision
    << ";ranks=" << p->rmax_a << "," << p->rmax_b << ";stages=" << p->n_stages << ";nrhs=" << nrhs;
  return o.str();
}

bool tune_cache_lookup(const char* path, const std::string& sig, fmm::Schedule& out) {
  std::ifstream f(path);
  std::string line;
  bool found = false;
  while (std::getline(f, line)) {
    std::istringstream is(line);
    std::string key;
    fmm::Schedule sc;
    double ms = 0;
    if ((is >> key >> sc.xrows >> sc.tc_slab >> sc.tc_gemm >> sc.no_overlap >> ms) && key == sig) {
      out = sc;
      found = true;   // the last entry for a signature wins
    }
  }
  return found;
}

}  // namespace

extern "C" {

int fmmfft_autotune(fmmfft_plan p, int nrhs, double budget_ms) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (!p->ready) return FMMFFT_ERR_NOT_COMPRESSED;
  if (nrhs < 1 || nrhs > 4096 || !(budget_ms > 0)) return FMMFFT_ERR_INVALID_ARG;
  const std::string sig = tune_signature(p, nrhs);
  const char* cache = std::getenv("FMMFFT_TUNE_CACHE");
  const fmm::Schedule before = p->sched;
  if (cache && *cache) {
    fmm::Schedule sc;
    if (tune_cache_lookup(cache, sig, sc)) {
      p->sched = sc;
      if (check_supported(p) && ensure_slabs(p) == FMMFFT_OK) return FMMFFT_OK;
      p->sched = before;   // stale entry: tune again
    }
  }
  // candidates, the current default first
  std::vector<fmm::Schedule> cand;
  const fmm::TranslateArgs a0 = base_args(p);
  const bool tc_slab_applies = fmm::tc_restore_applies(a0);
  const bool stages = p->n_stages > 0;
  for (int xr : {2, 1, 4})
    for (int ts : tc_slab_applies ? std::vector<int>{-1, 0} : std::vector<int>{-1})
      for (int tg : (stages && fmm::tc_kind(p->precision) != 0) ? std::vector<int>{-1, 0} : std::vector<int>{-1})
        for (int no : stages ? std::vector<int>{0, 1} : std::vector<int>{0}) {
          fmm::Schedule sc;
          sc.xrows = xr;
          sc.tc_slab = ts;
          sc.tc_gemm = tg;
          sc.no_overlap = no;
          cand.push_back(sc);
        }
  const size_t bytes = (size_t)p->n_dir * 2 * nrhs * p->K[0] * p->K[1] * p->K[2] * elem_bytes(p);
  void *din = nullptr, *dout = nullptr;
  int st = dev_alloc(&din, bytes);
  if (st == FMMFFT_OK) st = dev_alloc(&dout, bytes);
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (st == FMMFFT_OK && (cudaMemset(din, 0, bytes) != cudaSuccess ||
                          cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                          cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess))
    st = FMMFFT_ERR_CUDA;
  const bool profile = p->profile;
  p->profile = false;
  // the caller's stream and status word stay as they were: the timing runs on
  // a private stream, whose handle must not outlive this call in last_stream,
  // and a status bit raised by a candidate belongs to that candidate alone
  cudaStream_t caller_stream = p->last_stream;
  int prior_status = 0;
  if (st == FMMFFT_OK && p->d_status) {
    if (cudaStreamSynchronize(caller_stream) != cudaSuccess ||
        cudaMemcpy(&prior_status, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = FMMFFT_ERR_CUDA;
  }
  auto take_status = [&](int* word) -> bool {   // read and clear; false on a CUDA error
    *word = 0;
    if (!p->d_status) return true;
    return cudaStreamSynchronize(s) == cudaSuccess &&
           cudaMemcpy(word, p->d_status, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess &&
           cudaMemset(p->d_status, 0, sizeof(int)) == cudaSuccess;
  };
  fmm::Schedule best = before;
  float best_ms = 0.f;
  bool have = false;
  const auto t_start = std::chrono::steady_clock::now();
  for (size_t c = 0; st == FMMFFT_OK && c < cand.size(); ++c) {
    if (have && std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count() >
                    budget_ms)
      break;
    p->sched = cand[c];
    if (!check_supported(p) || ensure_slabs(p) != FMMFFT_OK) continue;
    int rs = FMMFFT_OK;
    for (int w = 0; w < 2 && rs == FMMFFT_OK; ++w) rs = fmmfft_translate(p, din, dout, nrhs, s);
    const int reps = 5;
    cudaEventRecord(e0, s);
    for (int r = 0; r < reps && rs == FMMFFT_OK; ++r) rs = fmmfft_translate(p, din, dout, nrhs, s);
    cudaEventRecord(e1, s);
    if (rs != FMMFFT_OK || cudaEventSynchronize(e1) != cudaSuccess) {
      cudaGetLastError();
      int ignored = 0;
      take_status(&ignored);
      continue;
    }
    // a candidate that tripped a device check (rank over its shared memory,
    // a tensor-core wait limit) is not a valid schedule, however fast
    int cand_status = 0;
    if (!take_status(&cand_status)) {
      st = FMMFFT_ERR_CUDA;
      break;
    }
    if (cand_status != 0) continue;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    ms /= reps;
    if (!have || ms < best_ms) {
      best = cand[c];
      best_ms = ms;
      have = true;
    }
  }
  p->profile = profile;
  p->sched = have ? best : before;
  if (st == FMMFFT_OK && (!check_supported(p) || ensure_slabs(p) != FMMFFT_OK)) st = FMMFFT_ERR_UNSUPPORTED;
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  p->last_stream = caller_stream;
  if (p->d_status && cudaMemcpy(p->d_status, &prior_status, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess &&
      st == FMMFFT_OK)
    st = FMMFFT_ERR_CUDA;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  free_dev(din);
  free_dev(dout);
  if (st == FMMFFT_OK && have && cache && *cache) {
    std::ofstream f(cache, std::ios::app);
    if (f) f << sig << " " << best.xrows << " " << best.tc_slab << " " << best.tc_gemm << " " << best.no_overlap << " "
             << best_ms << "\n";
  }
  return st;
}

int fmmfft_plan_destroy(fmmfft_plan p) {
  if (!p) return FMMFFT_ERR_INVALID_ARG;
  if (p->last_stream || p->d_status) cudaDeviceSynchronize();
  release_operator(p);
  free_dev(p->d_inter);
  free_dev(p->d_io);
  free_dev(p->d_weights);
  free_dev(p->d_occ);
  for (auto& ev : p->events)
    if (ev) cudaEventDestroy(ev);
  if (p->side) {
    cudaStreamSynchronize(p->side);
    cudaStreamDestroy(p->side);
  }
  if (p->fork) cudaEventDestroy(p->fork);
  if (p->join) cudaEventDestroy(p->join);
  if (p->h2d) {
    cudaStreamSynchronize(p->h2d);
    cudaStreamSynchronize(p->d2h);
    cudaStreamDestroy(p->h2d);
    cudaStreamDestroy(p->d2h);
  }
  for (auto& ev : p->hev)
    if (ev) cudaEventDestroy(ev);
  void* s = p->d_status;
  free_dev(s);
  delete p;
  return FMMFFT_OK;
}

}  // extern "C"
