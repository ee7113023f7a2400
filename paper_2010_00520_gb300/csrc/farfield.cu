// Aggregation (Eq. 4) and disaggregation (Eq. 6): the far-field steps on
// either side of the translation of Eq. 5.
//
//   aggregation     A[p][c][r][v] = sum_{i < nb} P[p][c][i][v] I[r][i][v]
//   disaggregation  y[r][i][v]    = sum_p w_p sum_{c in {theta, phi}} conj(P[p][c][i][v]) B[p][c][r][v]
//
// P holds the theta / phi far-field patterns P^+(k_p, b) of the nb basis
// functions of every box (Eq. 3; P^- is its conjugate, Sec. II.A), I the
// basis-function coefficients of nrhs right-hand sides, A and B field spectra
// in the layout of the translation ([p][c][r][v]), w_p the quadrature weights
// of the directions.  v = (z Ky + y) Kx + x runs over the Kx Ky Kz boxes.
//
// Both steps stream the patterns once from HBM and do a few complex
// multiply-adds per pattern element (about 2 flop per byte), so they are
// HBM-bound: consecutive threads take consecutive boxes, so every pattern,
// field and coefficient access of a warp is one coalesced transaction.
//   * aggregation: a block takes a tile of boxes and a range of directions;
//     the tile's coefficients for up to RT right-hand sides are staged once in
//     shared memory and reused for every direction of the range;
//   * disaggregation: a thread takes one box, up to IT basis functions and up
//     to RT right-hand sides and sums a quarter of the directions in
//     registers; the four CTAs of a thread-block cluster take the four
//     quarters of the same outputs and add their partial sums through
//     distributed shared memory in a fixed order (deterministic, no scratch
//     in HBM, and four times the blocks of one sum per thread, which left
//     the last wave of SMs two-thirds full).  The four warps of a block take
//     four basis-function groups of the same 32 boxes, so the spectra they
//     all read come from HBM once and from L1 after that.
#include <cooperative_groups.h>

#include "../../include/fmmfft.h"
#include "fft_core.cuh"
#include "plan_internal.h"

namespace fmm {

namespace cg = cooperative_groups;

namespace {

constexpr int kAggBoxes = 128;     // boxes per aggregation block (threads)
constexpr int kDisBoxes = 128;     // threads per disaggregation block
constexpr int kDisWarps = kDisBoxes / 32;   // basis-function groups per block
constexpr int kDisIT = 4;          // basis functions per disaggregation thread
constexpr int kDisSplit = 4;       // CTAs per cluster, each summing a quarter of the directions

template <typename R> struct FarTile;
// RT right-hand sides per thread; QR pattern rows (direction x polarisation)
// per aggregation step
template <> struct FarTile<float> { static constexpr int RT = 4, QR = 4; };
template <> struct FarTile<double> { static constexpr int RT = 2, QR = 4; };

template <typename R>
__global__ void __launch_bounds__(kAggBoxes, 3) aggregate_kernel(const cx<R>* __restrict__ P,
                                                              const cx<R>* __restrict__ I,
                                                              cx<R>* __restrict__ A, int64_t V, int nb,
                                                              int nrhs, int n_dir, int dirs_per_block) {
  using C = cx<R>;
  constexpr int RT = FarTile<R>::RT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* sI = reinterpret_cast<C*>(smem_raw);   // [RT][nb][kAggBoxes]
  const int t = threadIdx.x;
  const int64_t v = (int64_t)blockIdx.x * kAggBoxes + t;
  const int r0 = blockIdx.z * RT;
  const int nr = min(RT, nrhs - r0);
  for (int r = 0; r < RT; ++r)
    for (int i = 0; i < nb; ++i)
      sI[(r * nb + i) * kAggBoxes + t] =
          (r < nr && v < V) ? I[((int64_t)(r0 + r) * nb + i) * V + v] : czero<C>();
  __syncthreads();
  if (v >= V) return;
  const int p0 = blockIdx.y * dirs_per_block;
  const int p1 = min(n_dir, p0 + dirs_per_block);
  // two directions x two polarisations (4 pattern rows) per step, four basis
  // functions at a time: 16 independent pattern loads in flight per thread,
  // since the staged coefficients allow only about 12 warps per SM (8 rows
  // per step measured slower: 0.369 against 0.334 ms at 16 basis functions)
  constexpr int QR = FarTile<R>::QR;
  for (int p = p0; p < p1; p += QR / 2) {
    const int rows = min(QR, 2 * (p1 - p));
    const C* Pr = P + ((int64_t)p * 2 * nb) * V + v;   // row q = 2 (p' - p) + c starts at q nb V
    C acc[QR][RT];
#pragma unroll
    for (int q = 0; q < QR; ++q)
#pragma unroll
      for (int r = 0; r < RT; ++r) acc[q][r] = czero<C>();
    for (int i = 0; i < nb; i += 4) {
      C pv[QR][4];
#pragma unroll
      for (int q = 0; q < QR; ++q)
#pragma unroll
        for (int u = 0; u < 4; ++u)
          pv[q][u] = (q < rows && i + u < nb) ? Pr[((int64_t)q * nb + i + u) * V] : czero<C>();
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (i + u >= nb) break;
        C iv[RT];
#pragma unroll
        for (int r = 0; r < RT; ++r) iv[r] = sI[(r * nb + i + u) * kAggBoxes + t];
#pragma unroll
        for (int q = 0; q < QR; ++q)
#pragma unroll
          for (int r = 0; r < RT; ++r) cfma(acc[q][r], pv[q][u], iv[r]);
      }
    }
#pragma unroll
    for (int q = 0; q < QR; ++q) {
      if (q >= rows) break;
      C* Ac = A + ((int64_t)(p * 2 + q) * nrhs + r0) * V + v;
#pragma unroll
      for (int r = 0; r < RT; ++r)
        if (r < nr) Ac[(int64_t)r * V] = acc[q][r];
    }
  }
}

template <typename R>
__global__ void __cluster_dims__(kDisSplit, 1, 1) __launch_bounds__(kDisBoxes)
    disaggregate_kernel(const cx<R>* __restrict__ P, const cx<R>* __restrict__ B, const double* __restrict__ w,
                        cx<R>* __restrict__ y, int64_t V, int nb, int nrhs, int n_dir) {
  using C = cx<R>;
  constexpr int RT = FarTile<R>::RT;
  constexpr int NC = kDisIT * RT;               // outputs per thread
  __shared__ C part[NC][kDisBoxes];             // this CTA's partial sums
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank();      // which quarter of the directions
  // warp j of the block takes basis-function group gs * kDisWarps + j for the
  // same 32 boxes (one per lane): the warps of a block read the same spectra,
  // which the first one brings into this SM's L1
  const int groups = (nb + kDisIT - 1) / kDisIT;
  const int gsets = (groups + kDisWarps - 1) / kDisWarps;
  const int64_t unit = blockIdx.x / kDisSplit;
  const int gs = (int)(unit % gsets);
  const int64_t tile = unit / gsets;
  const int t = threadIdx.x;
  const int g = gs * kDisWarps + (t >> 5);
  const int64_t v = tile * 32 + (t & 31);
  const int i0 = g * kDisIT;
  const int ni = min(kDisIT, nb - i0);
  const bool live = v < V && ni > 0;
  const int r0 = blockIdx.y * RT;
  const int nr = min(RT, nrhs - r0);
  const int per = (n_dir + kDisSplit - 1) / kDisSplit;
  const int pa = s * per, pb = min(n_dir, pa + per);
  C acc[kDisIT][RT];
#pragma unroll
  for (int i = 0; i < kDisIT; ++i)
#pragma unroll
    for (int r = 0; r < RT; ++r) acc[i][r] = czero<C>();
  if (live && pa < pb) {
    // the next direction's patterns and spectra are loaded while the current
    // one is summed: 16 loads per thread in flight behind the arithmetic
    C pn[2][kDisIT], bn[2][RT];
    auto load = [&](int p) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const C* Bc = B + ((int64_t)(p * 2 + c) * nrhs + r0) * V + v;
        const C* Pc = P + ((int64_t)(p * 2 + c) * nb + i0) * V + v;
#pragma unroll
        for (int r = 0; r < RT; ++r) bn[c][r] = r < nr ? Bc[(int64_t)r * V] : czero<C>();
#pragma unroll
        for (int i = 0; i < kDisIT; ++i) pn[c][i] = i < ni ? Pc[(int64_t)i * V] : czero<C>();
      }
    };
    load(pa);
    for (int p = pa; p < pb; ++p) {
      C pc[2][kDisIT], b[2][RT];
#pragma unroll
      for (int c = 0; c < 2; ++c) {
#pragma unroll
        for (int i = 0; i < kDisIT; ++i) pc[c][i] = pn[c][i];
#pragma unroll
        for (int r = 0; r < RT; ++r) b[c][r] = bn[c][r];
      }
      if (p + 1 < pb) load(p + 1);
      const R wp = (R)w[p];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int i = 0; i < kDisIT; ++i) {
          const C q = mk<C>(wp * pc[c][i].x, -wp * pc[c][i].y);   // w_p conj(P)
#pragma unroll
          for (int r = 0; r < RT; ++r) cfma(acc[i][r], q, b[c][r]);
        }
    }
  }
#pragma unroll
  for (int i = 0; i < kDisIT; ++i)
#pragma unroll
    for (int r = 0; r < RT; ++r) part[i * RT + r][t] = acc[i][r];
  cluster.sync();
  // CTA s of the cluster finishes the outputs k = s, s + kDisSplit, ...: the
  // partial sums of the cluster's CTAs, read through distributed shared
  // memory and added in CTA order (deterministic)
  if (live) {
    for (int k = s; k < NC; k += kDisSplit) {
      const int i = k / RT, r = k % RT;
      if (i >= ni || r >= nr) continue;
      C sum = czero<C>();
#pragma unroll
      for (int q = 0; q < kDisSplit; ++q) {
        const C* rp = cluster.map_shared_rank(&part[k][t], q);
        sum = cadd(sum, *rp);
      }
      y[((int64_t)(r0 + r) * nb + i0 + i) * V + v] = sum;
    }
  }
  // no CTA may leave while another still reads its shared memory
  cluster.sync();
}

// ---------------------------------------------------------------------------
// Inverse x pass fused with the disaggregation: the translated fields B of
// Eq. 5 leave the last inverse DFT in shared memory and go straight into the
// sum of Eq. 6, so they are never written to (or read back from) HBM.
//
// A block owns a tile of TR whole (y, z) rows (TR Kx <= 128 boxes), kXdRT
// right-hand sides and kXdNB basis functions, and one of the kDisSplit
// quarters of the directions (the quarters of a tile are the CTAs of one
// cluster and add their partial sums through distributed shared memory in a
// fixed order, as the separate disaggregation does).  For each direction p of
// its quarter, in order: the x-spectra of its 2 x kXdRT x TR lines are loaded
// (for each x, the TR rows are contiguous), inverse-transformed along x
// (first Kx outputs kept), and every thread adds w_p conj(P) B for its box
// and its 8 basis functions over both polarisations.  Threads 0..127 take
// basis functions 0..7 of the chunk, threads 128..255 functions 8..15, each
// for the box t % 128 of the tile.
// ---------------------------------------------------------------------------
constexpr int kXdRT = 2;           // right-hand sides per block
constexpr int kXdNB = 16;          // basis functions per block
constexpr int kXdIT = 8;           // basis functions per thread
constexpr int kXdBoxes = 128;      // boxes per tile (at most)

template <typename R, int N1>
__global__ void __cluster_dims__(kDisSplit, 1, 1) __launch_bounds__(kThreads)
    xinv_disagg_kernel(const cx<R>* __restrict__ inter, const cx<R>* __restrict__ P,
                       const double* __restrict__ w, cx<R>* __restrict__ y, const cx<R>* __restrict__ twg,
                       const unsigned char* __restrict__ occ, const unsigned char* __restrict__ rowocc,
                       int Kx, int rows, int TR, int nb, int nrhs, int n_dir) {
  using C = cx<R>;
  using L = Line<N1>;
  constexpr int PX = N1 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xs = tw + N1;
  C* Q0 = xs + kWarps * L::XW;                   // two buffers of lines x PX (directions alternate)
  C* part = Q0;                                  // reused for the partial sums at the end
  cg::cluster_group cluster = cg::this_cluster();
  const int s = (int)cluster.block_rank();
  // blockIdx.x = (tile * rchunks + RHS chunk) * kDisSplit + quarter: the
  // blocks of one tile's RHS chunks are neighbours, so the patterns they all
  // read come from HBM once and from L2 after that
  const int rchunks = (nrhs + kXdRT - 1) / kXdRT;
  const int unit = blockIdx.x / kDisSplit;
  const int tile = unit / rchunks;
  const int r0 = tile * TR;
  const int nrow = min(TR, rows - r0);
  const int rh0 = (unit - tile * rchunks) * kXdRT;
  const int nr = min(kXdRT, nrhs - rh0);
  const int i0 = blockIdx.z * kXdNB;
  const int t = threadIdx.x;
  const int b = t % kXdBoxes, g = t / kXdBoxes;
  const int brow = b / Kx, bx = b - brow * Kx;
  // an empty box (occupancy mask) receives nothing: its B is zero, so are
  // its outputs
  const bool inb = brow < nrow;
  const bool live = inb && (!occ || occ[(int64_t)(r0 + brow) * Kx + bx]);
  const int64_t V = (int64_t)rows * Kx;
  const int64_t v = (int64_t)(r0 + brow) * Kx + bx;
  const int ia = i0 + g * kXdIT;
  const int ni = max(0, min(kXdIT, nb - ia));
  const int lines = 2 * kXdRT * TR;
  const int per = (n_dir + kDisSplit - 1) / kDisSplit;
  const int pa = s * per, pb = min(n_dir, pa + per);
  for (int i = t; i < N1; i += kThreads) tw[i] = twg[i];
  TeamPos<N1> tp;
  C* xt = tp.xs(xs);
  C acc[kXdIT][kXdRT];
#pragma unroll
  for (int i = 0; i < kXdIT; ++i)
#pragma unroll
    for (int r = 0; r < kXdRT; ++r) acc[i][r] = czero<C>();
  // line l = (c kXdRT + rr) TR + row of direction q's buffer holds field
  // ((q 2 + c) nrhs + rh0 + rr), row r0 + row: copied asynchronously
  // (cp.async), so that direction q + 1's lines arrive while q is
  // transformed and summed; lines of absent fields or empty rows are zeroed
  const int qbuf = lines * PX;
  auto issue = [&](int q, C* Qb) {
    for (int e = t; e < lines * N1; e += kThreads) {
      const int row = e % TR, rest = e / TR;
      const int x = rest % N1, cr = rest / N1;
      const int c = cr / kXdRT, rr = cr % kXdRT;
      C* dst = Qb + (cr * TR + row) * PX + x;
      if (rr < nr && row < nrow && (!rowocc || rowocc[r0 + row])) {
        const int64_t f = ((int64_t)(q * 2 + c) * nrhs + rh0 + rr);
        const C* src = inter + (f * N1 + x) * rows + r0 + row;
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                     "l"(src),
                     "n"((int)sizeof(C))
                     : "memory");
      } else {
        *dst = czero<C>();
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  if (pa < pb) issue(pa, Q0);
  for (int p = pa; p < pb; ++p) {
    C* Q = Q0 + ((p - pa) & 1) * qbuf;
    // patterns of this direction, issued before the transform so that their
    // latency overlaps it
    C pv[2][kXdIT];
#pragma unroll
    for (int c = 0; c < 2; ++c)
#pragma unroll
      for (int i = 0; i < kXdIT; ++i)
        pv[c][i] = (live && i < ni) ? P[((int64_t)(p * 2 + c) * nb + ia + i) * V + v] : czero<C>();
    // this direction's lines have landed (own copies), then everyone's
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    // the other buffer was last read in the previous iteration, before the
    // barrier above
    if (p + 1 < pb) issue(p + 1, Q0 + ((p + 1 - pa) & 1) * qbuf);
    for (int base = 0; base < lines; base += L::LPI) {
      const int ln = base + tp.line;
      const bool act = ln < lines;
      line_fft<N1, +1, false>(Q + (act ? ln : 0) * PX, 1, xt, tw, tp.t, act, Kx);
    }
    __syncthreads();
    const R wp = (R)w[p];
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      C bv[kXdRT];
#pragma unroll
      for (int rr = 0; rr < kXdRT; ++rr)
        bv[rr] = live ? Q[((c * kXdRT + rr) * TR + brow) * PX + bx] : czero<C>();
#pragma unroll
      for (int i = 0; i < kXdIT; ++i) {
        const C q = mk<C>(wp * pv[c][i].x, -wp * pv[c][i].y);    // w_p conj(P)
#pragma unroll
        for (int rr = 0; rr < kXdRT; ++rr) cfma(acc[i][rr], q, bv[rr]);
      }
    }
  }
  __syncthreads();                               // Q no longer read
#pragma unroll
  for (int i = 0; i < kXdIT; ++i)
#pragma unroll
    for (int rr = 0; rr < kXdRT; ++rr) part[(i * kXdRT + rr) * kThreads + t] = acc[i][rr];
  cluster.sync();
  // CTA s finishes the outputs k = s, s + kDisSplit, ... in CTA order
  if (inb) {
    for (int k = s; k < kXdIT * kXdRT; k += kDisSplit) {
      const int i = k / kXdRT, rr = k % kXdRT;
      if (i >= ni || rr >= nr) continue;
      C sum = czero<C>();
#pragma unroll
      for (int q = 0; q < kDisSplit; ++q) {
        const C* rp = cluster.map_shared_rank(&part[k * kThreads + t], q);
        sum = cadd(sum, *rp);
      }
      y[((int64_t)(rh0 + rr) * nb + ia + i) * V + v] = sum;
    }
  }
  cluster.sync();
}

// Tile rows and shared memory of the fused kernel.
template <typename R, int N1>
size_t xinv_disagg_smem(int TR) {
  const size_t q = (size_t)2 * 2 * kXdRT * TR * (N1 + 1);     // two line buffers
  const size_t part = (size_t)kXdIT * kXdRT * kThreads;
  return sizeof(cx<R>) * (N1 + kWarps * Line<N1>::XW + (q > part ? q : part));
}

template <typename R, int N1>
cudaError_t xinv_disagg_t(const XDisArgs& a) {
  if (a.Kx > kXdBoxes || a.Kx < 1) return cudaErrorInvalidValue;
  const int TR = kXdBoxes / a.Kx;
  const int tiles = (a.rows + TR - 1) / TR;
  const int rchunks = (a.nrhs + kXdRT - 1) / kXdRT;
  const int nchunks = (a.nb + kXdNB - 1) / kXdNB;
  if ((int64_t)tiles * rchunks * kDisSplit > 0x7fffffff || nchunks > 65535) return cudaErrorInvalidValue;
  const size_t smem = xinv_disagg_smem<R, N1>(TR);
  static std::atomic<int> optin[kMaxDevices];
  auto kern = xinv_disagg_kernel<R, N1>;
  cudaError_t e = smem_optin((const void*)kern, optin);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)((int64_t)tiles * rchunks * kDisSplit), 1, nchunks), kThreads, smem, a.stream>>>(
      (const cx<R>*)a.inter, (const cx<R>*)a.P, a.w, (cx<R>*)a.y, (const cx<R>*)a.tw, a.occ, a.rowocc, a.Kx,
      a.rows, TR, a.nb, a.nrhs, a.n_dir);
  return cudaGetLastError();
}

template <typename R>
cudaError_t xinv_disagg_any(const XDisArgs& a) {
  switch (a.n1) {
    case 4: return xinv_disagg_t<R, 4>(a);
    case 8: return xinv_disagg_t<R, 8>(a);
    case 16: return xinv_disagg_t<R, 16>(a);
    case 32: return xinv_disagg_t<R, 32>(a);
    case 64: return xinv_disagg_t<R, 64>(a);
    case 128: return xinv_disagg_t<R, 128>(a);
    case 256: return xinv_disagg_t<R, 256>(a);
    default: return cudaErrorInvalidValue;
  }
}

template <typename R>
cudaError_t aggregate_t(const FarFieldArgs& a) {
  constexpr int RT = FarTile<R>::RT;
  const int64_t tiles = (a.V + kAggBoxes - 1) / kAggBoxes;
  const int rchunks = (a.nrhs + RT - 1) / RT;
  // enough blocks for a few waves of 152 SMs, each spanning as many directions
  // as that leaves, so that the staged coefficients are reused
  const int64_t want = 152 * 8;
  int64_t split = (want + tiles * rchunks - 1) / (tiles * rchunks);
  split = split < 1 ? 1 : (split > a.n_dir ? a.n_dir : split);
  const int dirs = (int)((a.n_dir + split - 1) / split);
  const int ychunks = (a.n_dir + dirs - 1) / dirs;
  const size_t smem = (size_t)RT * a.nb * kAggBoxes * sizeof(cx<R>);
  if (tiles > 0x7fffffff || ychunks > 65535 || rchunks > 65535) return cudaErrorInvalidValue;
  static std::atomic<int> optin[kMaxDevices];
  auto kern = aggregate_kernel<R>;
  cudaError_t e = smem_optin((const void*)kern, optin);
  if (e != cudaSuccess) return e;
  kern<<<dim3((unsigned)tiles, ychunks, rchunks), kAggBoxes, smem, a.stream>>>(
      (const cx<R>*)a.P, (const cx<R>*)a.in, (cx<R>*)a.out, a.V, a.nb, a.nrhs, a.n_dir, dirs);
  return cudaGetLastError();
}

template <typename R>
cudaError_t disaggregate_t(const FarFieldArgs& a) {
  constexpr int RT = FarTile<R>::RT;
  const int64_t tiles = (a.V + 31) / 32;
  const int groups = (a.nb + kDisIT - 1) / kDisIT;
  const int gsets = (groups + kDisWarps - 1) / kDisWarps;
  const int rchunks = (a.nrhs + RT - 1) / RT;
  if (tiles * gsets * kDisSplit > 0x7fffffff || rchunks > 65535) return cudaErrorInvalidValue;
  disaggregate_kernel<R><<<dim3((unsigned)(tiles * gsets * kDisSplit), rchunks), kDisBoxes, 0, a.stream>>>(
      (const cx<R>*)a.P, (const cx<R>*)a.in, a.w, (cx<R>*)a.out, a.V, a.nb, a.nrhs, a.n_dir);
  return cudaGetLastError();
}

}  // namespace

size_t aggregate_smem_bytes(int nb, bool fp64) {
  return fp64 ? (size_t)FarTile<double>::RT * nb * kAggBoxes * sizeof(double2)
              : (size_t)FarTile<float>::RT * nb * kAggBoxes * sizeof(float2);
}

cudaError_t launch_aggregate(const FarFieldArgs& a) {
  if (a.V == 0 || a.n_dir == 0) return cudaSuccess;
  return a.fp64 ? aggregate_t<double>(a) : aggregate_t<float>(a);
}

cudaError_t launch_disaggregate(const FarFieldArgs& a) {
  if (a.V == 0) return cudaSuccess;
  return a.fp64 ? disaggregate_t<double>(a) : disaggregate_t<float>(a);
}

cudaError_t launch_xinv_disaggregate(const XDisArgs& a) {
  if (a.rows == 0 || a.Kx == 0) return cudaSuccess;
  return a.fp64 ? xinv_disagg_any<double>(a) : xinv_disagg_any<float>(a);
}

}  // namespace fmm
