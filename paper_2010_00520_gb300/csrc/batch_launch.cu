// Shared launches of a batch of translations (many independent FMM-FFT
// instances of uneven grids, ranks and RHS counts; Sec. II.C per instance):
// the instances are grouped into shape classes (FFT extents, operator kind,
// restore arithmetic) and every phase runs one launch per class over the
// work items of all the class's instances, instead of one launch per
// instance:
//
//   pre-pass  the restore products of every instance (the steps of Figs. 3-4
//             that do not depend on x), one batched-GEMM launch per stage
//             index and arithmetic, their descriptors gathered into one array;
//   x fwd     per class: items (instance, field, row block);
//   yz        per class: items (instance, x, direction), slab restore and
//             the y/z transforms with the Hadamard product;
//   x inv     per class, as x fwd.
//
// The classes run on separate streams forked from the caller's, so that one
// class's HBM-bound x passes overlap another's arithmetic-bound yz pass.  The
// kernels are the single-translation kernels in their batch mode
// (translate_kernels.cuh): a block looks up its items' instance parameters
// and runs the same per-item code, so a batched translation equals the
// instances' own translations bit for bit.
#include <algorithm>
#include <cstring>
#include <map>
#include <tuple>

#include "translate_kernels.cuh"

namespace fmm {

cudaError_t launch_x_batch(bool fwd, int n1, const BatchXTable& T, long long total, size_t smem, cudaStream_t s);
void x_pass_shape(int n1, int rows, int mult, int* rpb, size_t* smem);
cudaError_t launch_yz_batch(int fmt, const YZParams& P, int n2, int n3, size_t smem, cudaStream_t s,
                            const BatchYZ* inst, int ninst, long long total);

namespace {

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// One x-pass launch per kXTable instances of a class, each with its
// instances' descriptors as launch parameters (items renumbered from 0).
cudaError_t x_tables(bool fwd, int n1, const std::vector<BatchX>& d, long long total, size_t smem, cudaStream_t s) {
  for (size_t i0 = 0; i0 < d.size(); i0 += kXTable) {
    const size_t n = std::min<size_t>(kXTable, d.size() - i0);
    BatchXTable T;
    std::memset(&T, 0, sizeof(T));
    const long long first = d[i0].item0;
    const long long end = i0 + n < d.size() ? d[i0 + n].item0 : total;
    for (size_t j = 0; j < n; ++j) {
      T.inst[j] = d[i0 + j];
      T.inst[j].item0 -= first;
    }
    T.ninst = (int)n;
    cudaError_t e = launch_x_batch(fwd, n1, T, end - first, smem, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

struct Class {
  std::vector<BatchX> fwd, inv;
  long long x_total = 0;
  size_t x_smem = 0;
  std::vector<BatchYZ> yz;
  long long yz_total = 0;
  size_t yz_smem = 0;
};

}  // namespace

bool batch_persistent_ok(const TranslateArgs& a) {
  const bool prec_ok = a.precision != FMMFFT_PREC_C128;
  return prec_ok && !a.large && a.p0 == 0 && a.nw == 0 && a.dis == nullptr && a.yz_fmt >= 0 && a.yz_fmt <= 2;
}

cudaError_t launch_translate_batch(const std::vector<TranslateArgs>& args, BatchDev& dev, cudaStream_t s,
                                   const std::vector<cudaStream_t>& lanes) {
  const int n = (int)args.size();
  if (n == 0) return cudaSuccess;
  // classes by (n1, n2, n3, yz_fmt, tc)
  std::map<std::tuple<int, int, int, int, int>, Class> cls;
  for (int i = 0; i < n; ++i) {
    const TranslateArgs& a = args[i];
    const int rows = a.K[1] * a.K[2];
    const int F = a.n_dir * 2 * a.nrhs;
    XPassParams X;
    std::memset(&X, 0, sizeof(X));
    X.tw = a.tw[0];
    X.Kx = a.K[0];
    X.rows = rows;
    size_t xs = 0;
    x_pass_shape(a.n[0], rows, a.xrows, &X.rows_per_block, &xs);
    if (X.rows_per_block <= 0) return cudaErrorInvalidValue;
    X.occ = a.occ;
    X.rowocc = a.rowocc;
    Class& c = cls[std::make_tuple(a.n[0], a.n[1], a.n[2], a.yz_fmt, a.tc)];
    // every byte defined (the descriptors are compared bytewise between calls)
    BatchX f, v;
    std::memset(&f, 0, sizeof(f));
    std::memset(&v, 0, sizeof(v));
    f.P = X;
    f.P.src = a.s_in;
    f.P.dst = a.inter;
    f.item0 = c.x_total;
    v.P = X;
    v.P.src = a.inter;
    v.P.dst = a.s_out;
    v.item0 = c.x_total;
    c.fwd.push_back(f);
    c.inv.push_back(v);
    c.x_total += (long long)F * ((rows + X.rows_per_block - 1) / X.rows_per_block);
    if (X.occ && X.rowocc) xs += xpass_mask_bytes(X.rows_per_block, X.Kx);
    c.x_smem = std::max(c.x_smem, xs);
    BatchYZ b;
    std::memset(&b, 0, sizeof(b));
    YZParams& Y = b.P;
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
    Y.n_dir = a.n_dir;
    Y.p0 = 0;
    b.item0 = c.yz_total;
    c.yz.push_back(b);
    c.yz_total += (long long)a.n[0] * a.n_dir;
    c.yz_smem = std::max(c.yz_smem, yz_smem_bytes(a));
  }
  // pre-pass products of every compressed instance, merged per stage index
  // and arithmetic (tensor cores in 3xTF32 / TF32 or BF16x3, or CUDA cores)
  struct Merge {
    int stage, tc_gemm, single;
    std::vector<std::pair<const GemmDesc*, int>> parts;
    int max_m = 0, max_n = 0, batch = 0;
    int* status = nullptr;
  };
  std::vector<Merge> merges;
  for (int i = 0; i < n; ++i) {
    const TranslateArgs& a = args[i];
    if (!a.prepass) continue;
    for (int k = 0; k < a.n_stages; ++k) {
      const int tg = a.tc_gemm;
      const int single = tg == 1 ? a.tc_single : 0;
      Merge* m = nullptr;
      for (auto& mm : merges)
        if (mm.stage == k && mm.tc_gemm == tg && mm.single == single) m = &mm;
      if (!m) {
        merges.push_back(Merge{k, tg, single, {}, 0, 0, 0, a.status});
        m = &merges.back();
      }
      m->parts.push_back({a.stages[k].desc, a.stages[k].batch});
      m->max_m = std::max(m->max_m, a.stages[k].max_m);
      m->max_n = std::max(m->max_n, a.stages[k].max_n);
      m->batch += a.stages[k].batch;
    }
  }
  std::stable_sort(merges.begin(), merges.end(), [](const Merge& u, const Merge& v) { return u.stage < v.stage; });
  // one device buffer: every class's descriptors, then the pre-pass products
  std::vector<unsigned char> host;
  auto put = [&](const void* p, size_t bytes) {
    const size_t at = align_up(host.size(), 256);
    host.resize(at + bytes);
    std::memcpy(host.data() + at, p, bytes);
    return at;
  };
  // (the x passes' descriptors travel as launch parameters)
  std::vector<size_t> off;
  for (auto& kv : cls) off.push_back(put(kv.second.yz.data(), sizeof(BatchYZ) * kv.second.yz.size()));
  size_t n_gemm = 0;
  for (auto& m : merges) n_gemm += m.batch;
  const size_t o_gm = align_up(host.size(), 256);
  const size_t bytes = o_gm + sizeof(GemmDesc) * std::max<size_t>(n_gemm, 1);
  host.resize(o_gm);
  // the gathered pre-pass descriptors are copied device to device; their
  // source addresses stand in for them in the change check
  std::vector<const void*> gsrc;
  for (auto& m : merges)
    for (auto& pr : m.parts) gsrc.push_back(pr.first);
  cudaError_t e;
  if (!dev.pre && (e = cudaEventCreateWithFlags(&dev.pre, cudaEventDisableTiming)) != cudaSuccess) return e;
  if (host != dev.host || gsrc != dev.gemm_src) {
    // the batch's launches in flight read the old descriptors
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
    for (auto l : lanes)
      if ((e = cudaStreamSynchronize(l)) != cudaSuccess) return e;
    if (bytes > dev.bytes) {
      if (dev.d_desc) cudaFree(dev.d_desc);
      dev.d_desc = nullptr;
      dev.bytes = 0;
      if ((e = cudaMalloc(&dev.d_desc, bytes)) != cudaSuccess) return e;
      dev.bytes = bytes;
    }
    if (!host.empty() && (e = cudaMemcpy(dev.d_desc, host.data(), host.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
      return e;
    size_t at = 0;
    for (auto& m : merges)
      for (auto& pr : m.parts) {
        if ((e = cudaMemcpy((char*)dev.d_desc + o_gm + sizeof(GemmDesc) * at, pr.first, sizeof(GemmDesc) * pr.second,
                            cudaMemcpyDeviceToDevice)) != cudaSuccess)
          return e;
        at += pr.second;
      }
    dev.host = host;
    dev.gemm_src = gsrc;
  }
  const char* base = (const char*)dev.d_desc;
  // pre-pass, one launch per merged stage (a device failure is reported on
  // the plan of the stage's first instance)
  {
    static std::atomic<int> optin_t[kMaxDevices], optin_b[kMaxDevices];
    if ((e = smem_optin((const void*)cgemm_batched_tc_kernel<false>, optin_t)) != cudaSuccess) return e;
    if ((e = smem_optin((const void*)cgemm_batched_tc_kernel<true>, optin_b)) != cudaSuccess) return e;
    size_t at = 0;
    for (auto& m : merges) {
      const GemmDesc* d = (const GemmDesc*)(base + o_gm) + at;
      dim3 grid((m.max_n + kGemmT - 1) / kGemmT, (m.max_m + kGemmT - 1) / kGemmT, m.batch);
      if (m.tc_gemm == 2) cgemm_batched_tc_kernel<true><<<grid, kThreads, kTcGemmSmem, s>>>(d, m.status, 0);
      else if (m.tc_gemm == 1)
        cgemm_batched_tc_kernel<false><<<grid, kThreads, kTcGemmSmem, s>>>(d, m.status, m.single);
      else cgemm_batched_kernel<float><<<grid, kThreads, 0, s>>>(d);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      at += m.batch;
    }
  }
  // every class waits for the merged pre-pass, then runs its three phases
  // on its lane
  if ((e = cudaEventRecord(dev.pre, s)) != cudaSuccess) return e;
  for (auto l : lanes)
    if ((e = cudaStreamWaitEvent(l, dev.pre, 0)) != cudaSuccess) return e;
  size_t k = 0;
  for (auto& kv : cls) {
    const Class& c = kv.second;
    const int n1 = std::get<0>(kv.first), n2 = std::get<1>(kv.first), n3 = std::get<2>(kv.first);
    const int fmt = std::get<3>(kv.first);
    cudaStream_t l = lanes.empty() ? s : lanes[k % lanes.size()];
    if ((e = x_tables(true, n1, c.fwd, c.x_total, c.x_smem, l)) != cudaSuccess) return e;
    if ((e = launch_yz_batch(fmt, c.yz[0].P, n2, n3, c.yz_smem, l, (const BatchYZ*)(base + off[k]),
                             (int)c.yz.size(), c.yz_total)) != cudaSuccess)
      return e;
    if ((e = x_tables(false, n1, c.inv, c.x_total, c.x_smem, l)) != cudaSuccess) return e;
    ++k;
  }
  return cudaSuccess;
}

void batch_dev_release(BatchDev& dev) {
  if (dev.pre) cudaEventDestroy(dev.pre);
  dev.pre = nullptr;
  if (dev.d_desc) cudaFree(dev.d_desc);
  dev.d_desc = nullptr;
  dev.bytes = 0;
  dev.host.clear();
  dev.gemm_src.clear();
}

}  // namespace fmm
