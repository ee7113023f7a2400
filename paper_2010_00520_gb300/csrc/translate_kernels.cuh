// Kernels of the translation stage (Eq. 5) and of the operator restorations
// (Sec. II.C, Figs. 3 and 4).
//
// A field A (Kz x Ky x Kx, x fastest) is translated in three passes:
//   xfwd  : rows r = z Ky + y: zero-pad x to n1, forward DFT along x, write
//           the x-spectrum transposed to the intermediate I[f][x][r]
//   yz    : one block per (x, direction p): the operator slab T~_p[x][:][:]
//           is loaded (format NONE) or restored (compressed formats) into
//           shared memory once, then for every field of direction p: forward
//           DFT along y (rows z < Kz), along z (columns) fused with the
//           Hadamard product and the inverse DFT along z, inverse DFT along y,
//           and the Kz x Ky corner is written back in place
//   xinv  : inverse DFT along x of every row, first Kx entries written out
// The 1 / (n1 n2 n3) of the inverse transform is folded into the operator.
//
// Restoration is split between a pre-pass and the yz kernel.  The pre-pass
// (batched complex GEMMs, `cgemm_batched_kernel`) forms per call what does not
// depend on x: the core of each direction for the 4D formats (Figs. 3(b),
// 3(c), 4(b)) and H = U1 . mat(core), an n1 x (...) matrix whose row x is all
// the yz block (x, p) needs besides two small factor matrices:
//   Tucker-like (Tucker-3D, Tucker-4D, H-Tucker):
//       slab[z][y] = sum_c U3[z][c] sum_b U2[y][b] H_p[x][b][c]
//   TT-like (TT-3D, TT-4D):
//       slab[z][y] = sum_b R_p[z][b] T1[x][y][b]
// with R_p = U3 of the direction (TT-3D) or the generated slice S_p^T (TT-4D).
#pragma once

#include <type_traits>

#include "fft_core.cuh"
#include "plan_internal.h"
#include "tc_cgemm.cuh"

namespace fmm {

// Status-word bits set by kernels instead of faulting.
enum : int {
  kStatusRankOverflow = 1,   // a direction's ranks exceed the launch's shared memory
  kStatusBadShape = 2,       // launch shape does not match the problem
  kStatusTcTimeout = 4,      // a tensor-core wait ran out of polls
};

struct XPassParams {
  const void* src;   // xfwd: S_in; xinv: intermediate
  void* dst;         // xfwd: intermediate; xinv: S_out
  const void* tw;    // W_n1^m table
  int Kx, rows;      // rows = Ky * Kz per field
  int rows_per_block;
  // box occupancy or null: empty boxes are read as zero (xfwd) and written as
  // zero (xinv); x-lines with no occupied box are neither read nor
  // transformed (xfwd writes their zero spectra, xinv their zero outputs)
  const unsigned char* occ;
  const unsigned char* rowocc;
};

struct YZParams {
  void* inter;       // [F][n1][Kz][Ky]
  const void* tw2, *tw3;
  int Ky, Kz, n1, nf;  // nf = fields per direction (2 nrhs)
  const void* op;      // plain: [p][x][z][y], scaled
  const SlabDesc* desc;
  double scale;        // restore scale 1 / (n1 n2 n3)
  int rmax_a, rmax_b;  // shared-memory capacity of the launch (ranks)
  int* status;
  int tc;              // restore on the tensor cores (TcRestore): 1 3xTF32, 2 BF16x3
  int tc_single;       // with tc == 1: one TF32 product instead of three
  int n_dir;           // directions of this launch: p0 .. p0 + n_dir - 1
  int p0;
  void* slab_scratch;  // large planes: one slot of slot_elems per block
  long long slot_elems;
};

// Batch mode of the x and yz kernels (batch_launch.cu): one launch covers
// the work items of several instances of one shape class, items item0 ..
// next item0 - 1 belonging to the instance; a block finds its item's
// instance by bisection, takes its parameters and runs the same per-item
// code as a single translation.
struct BatchX {
  XPassParams P;
  long long item0;
};
struct BatchYZ {
  YZParams P;
  long long item0;
};

template <typename D>
__device__ __forceinline__ int find_instance(const D* inst, int ninst, long long item) {
  int lo = 0, hi = ninst - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (inst[mid].item0 <= item) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// Plans whose restore can run on the tensor cores (3xTF32 or BF16x3):
// complex64, planes of 32 or 64 per side or multiples of 64, and (checked on
// the host) for the Tucker-like format at most 64 columns of H_p[x].
template <typename R, int N2, int N3, int FMT>
struct TcRestore {
  // 64-multiples (tiled over larger planes), or planes of 32 and 64 that one
  // partly filled 64 x 64 tile covers
  static constexpr bool available = sizeof(R) == 4 && FMT != 0 &&
                                    ((N2 % 64 == 0 && N3 % 64 == 0) ||
                                     (N2 % 32 == 0 && N3 % 32 == 0 && N2 <= 64 && N3 <= 64));
};

// ---------------------------------------------------------------------------
// x passes
// ---------------------------------------------------------------------------
// One element copied from global to shared memory asynchronously (cp.async,
// 8 or 16 bytes, both addresses aligned to the element size); cp_async_drain
// waits for all of this thread's copies.
template <typename C>
__device__ __forceinline__ void cp_async_elem(C* dst_smem, const C* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst_smem)),
               "l"(src), "n"((int)sizeof(C))
               : "memory");
}
__device__ __forceinline__ void cp_async_drain() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// With an occupancy mask an x-pass block stages its rows' flags after Q in
// its dynamic shared memory: one byte per x-line (live[r]), then the box
// flags of its rows (box[r Kx + x]).  Bytes, 16-byte multiple:
inline size_t xpass_mask_bytes(int rows_per_block, int Kx) {
  return ((size_t)rows_per_block * (1 + (size_t)Kx) + 15) / 16 * 16;
}

// Work item `item` (field item / row blocks, row block item % row blocks) of
// the forward x pass, by the whole block; `smem_raw` holds xpass_smem bytes.
template <typename R, int N1>
__device__ __forceinline__ void xfwd_body(const XPassParams& P, int item, unsigned char* smem_raw) {
  using C = cx<R>;
  using L = Line<N1>;
  constexpr int PX = N1 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xs = tw + N1;
  C* Q = xs + kWarps * L::XW;
  const int nrb = (P.rows + P.rows_per_block - 1) / P.rows_per_block;
  const int f = item / nrb;
  const int r0 = (item - f * nrb) * P.rows_per_block;
  const int nr = min(P.rows_per_block, P.rows - r0);
  const C* src = reinterpret_cast<const C*>(P.src) + ((size_t)f * P.rows + r0) * P.Kx;
  C* dst = reinterpret_cast<C*>(P.dst);
  for (int i = threadIdx.x; i < N1; i += kThreads) tw[i] = reinterpret_cast<const C*>(P.tw)[i];
  // occupancy mask: the block's x-line and box flags staged once (empty
  // boxes read as zero; empty x-lines are not transformed and their spectra
  // are written as zeros)
  const bool masked = P.occ && P.rowocc;
  unsigned char* live = reinterpret_cast<unsigned char*>(Q + (size_t)P.rows_per_block * PX);
  unsigned char* box = live + P.rows_per_block;
  if (masked) {
    for (int i = threadIdx.x; i < nr; i += kThreads) live[i] = P.rowocc[r0 + i];
    for (int i = threadIdx.x; i < nr * P.Kx; i += kThreads) box[i] = P.occ[(size_t)r0 * P.Kx + i];
    __syncthreads();
  }
  const int half = N1 / 2;
  // batches of kLd loads per thread are issued before their shared-memory
  // stores, so that several global loads are in flight per thread (the rows
  // are contiguous here; asynchronous copies measured slower).  The mask
  // test is a compile-time branch of its own, so that the unmasked loads
  // stay batched.
  constexpr int kLd = 8;
  auto load_rows = [&](auto mask_tag) {
    constexpr bool kMask = decltype(mask_tag)::value;
    for (int i0 = threadIdx.x; i0 < nr * half; i0 += kLd * kThreads) {
      C v[kLd];
#pragma unroll
      for (int j = 0; j < kLd; ++j) {
        const int i = i0 + j * kThreads;
        const int r = i / half, x = i - r * half;
        const bool in = i < nr * half && x < P.Kx && (!kMask || box[r * P.Kx + x]);
        v[j] = in ? src[(size_t)r * P.Kx + x] : czero<C>();
      }
#pragma unroll
      for (int j = 0; j < kLd; ++j) {
        const int i = i0 + j * kThreads;
        const int r = i / half, x = i - r * half;
        if (i < nr * half) Q[r * PX + x] = v[j];
      }
    }
  };
  if (masked) load_rows(std::true_type{});
  else load_rows(std::false_type{});
  __syncthreads();
  TeamPos<N1> tp;
  C* xt = tp.xs(xs);
  for (int base = 0; base < nr; base += L::LPI) {
    const int line = base + tp.line;
    const bool act = line < nr && (!masked || live[line]);
    line_fft<N1, -1, true>(Q + (line < nr ? line : 0) * PX, 1, xt, tw, tp.t, act, N1);
  }
  __syncthreads();
  // I[f][x][r]: rows contiguous for fixed x; a line with no occupied box has
  // a zero spectrum.  (x, r) from the element number by shift and mask over
  // the power of two rp2 >= rows per block (no division per element)
  const int lg = 31 - __clz(P.rows_per_block) + ((P.rows_per_block & (P.rows_per_block - 1)) ? 1 : 0);
  const int rp2 = 1 << lg;
  for (int i = threadIdx.x; i < (N1 << lg); i += kThreads) {
    const int x = i >> lg, r = i & (rp2 - 1);
    if (r >= nr) continue;
    const bool rl = !masked || live[r];
    dst[((size_t)f * N1 + x) * P.rows + r0 + r] = rl ? Q[r * PX + x] : czero<C>();
  }
}

template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xfwd_kernel(XPassParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xfwd_body<R, N1>(P, blockIdx.x, smem_raw);
}

// Batch mode of the x passes: block b takes item b of the launch's items,
// as a single translation's x pass does.  The instances' parameters travel
// in the launch's own parameter space (constant bank), like a single
// translation's, so the lookup is a few cached constant reads and the item
// code reads its parameters from the same space; a class with more than
// kXTable instances runs one launch per kXTable of them.
constexpr int kXTable = 96;
struct BatchXTable {
  BatchX inst[kXTable];        // item0 relative to the launch's first item
  int ninst;
};

template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xfwd_batch_kernel(const __grid_constant__ BatchXTable T) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long item = blockIdx.x;
  const int i = find_instance(T.inst, T.ninst, item);
  xfwd_body<R, N1>(T.inst[i].P, (int)(item - T.inst[i].item0), smem_raw);
}

// Work item `item` of the inverse x pass (as xfwd_body).
template <typename R, int N1>
__device__ __forceinline__ void xinv_body(const XPassParams& P, int item, unsigned char* smem_raw) {
  using C = cx<R>;
  using L = Line<N1>;
  constexpr int PX = N1 + 1;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xs = tw + N1;
  C* Q = xs + kWarps * L::XW;
  const int nrb = (P.rows + P.rows_per_block - 1) / P.rows_per_block;
  const int f = item / nrb;
  const int r0 = (item - f * nrb) * P.rows_per_block;
  const int nr = min(P.rows_per_block, P.rows - r0);
  const C* src = reinterpret_cast<const C*>(P.src);
  C* dst = reinterpret_cast<C*>(P.dst) + ((size_t)f * P.rows + r0) * P.Kx;
  for (int i = threadIdx.x; i < N1; i += kThreads) tw[i] = reinterpret_cast<const C*>(P.tw)[i];
  // occupancy mask: the block's x-line and box flags staged once (empty
  // x-lines are neither read nor transformed; empty boxes are written as
  // zeros)
  const bool masked = P.occ && P.rowocc;
  unsigned char* live = reinterpret_cast<unsigned char*>(Q + (size_t)P.rows_per_block * PX);
  unsigned char* box = live + P.rows_per_block;
  if (masked) {
    for (int i = threadIdx.x; i < nr; i += kThreads) live[i] = P.rowocc[r0 + i];
    for (int i = threadIdx.x; i < nr * P.Kx; i += kThreads) box[i] = P.occ[(size_t)r0 * P.Kx + i];
    __syncthreads();
  }
  // (x, r) by shift and mask over the power of two rp2 >= rows per block;
  // every load of the block issued at once as an asynchronous copy into its
  // place in Q, then drained: the block reads n1 runs of its rows, one per
  // x, and the more of them in flight the better (128x128x32 boxes: 10.85
  // -> 9.15 ms against batches of eight register loads per thread)
  const int lg = 31 - __clz(P.rows_per_block) + ((P.rows_per_block & (P.rows_per_block - 1)) ? 1 : 0);
  const int rp2 = 1 << lg;
  for (int i = threadIdx.x; i < (N1 << lg); i += kThreads) {
    const int x = i >> lg, r = i & (rp2 - 1);
    if (r >= nr || (masked && !live[r])) continue;      // an empty line is not transformed
    cp_async_elem(Q + r * PX + x, src + ((size_t)f * N1 + x) * P.rows + r0 + r);
  }
  cp_async_drain();
  __syncthreads();
  TeamPos<N1> tp;
  C* xt = tp.xs(xs);
  for (int base = 0; base < nr; base += L::LPI) {
    const int line = base + tp.line;
    const bool act = line < nr && (!masked || live[line]);
    line_fft<N1, +1, false>(Q + (line < nr ? line : 0) * PX, 1, xt, tw, tp.t, act, P.Kx);
  }
  __syncthreads();
  // one row per warp at a time, lanes along x (coalesced, no division)
  const int lane = threadIdx.x & 31;
  for (int r = threadIdx.x >> 5; r < nr; r += kWarps)
    for (int x = lane; x < P.Kx; x += 32) {
      const bool occupied = !masked || box[r * P.Kx + x];
      dst[(size_t)r * P.Kx + x] = occupied ? Q[r * PX + x] : czero<C>();
    }
}

template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xinv_kernel(XPassParams P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  xinv_body<R, N1>(P, blockIdx.x, smem_raw);
}

template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xinv_batch_kernel(const __grid_constant__ BatchXTable T) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long item = blockIdx.x;                 // as in xfwd_batch_kernel
  const int i = find_instance(T.inst, T.ninst, item);
  xinv_body<R, N1>(T.inst[i].P, (int)(item - T.inst[i].item0), smem_raw);
}

// Shared memory of the x passes (bytes).
template <typename R, int N1>
constexpr size_t xpass_smem(int rows_per_block) {
  return sizeof(cx<R>) * (N1 + kWarps * Line<N1>::XW + (size_t)rows_per_block * (N1 + 1));
}

// Rows per x-pass block: `mult` (1, 2, 4; 0 = 2) times the lines one block
// iteration covers, halved while the shared memory exceeds 96 KB, at most
// the rows of a field.
template <typename R, int N1>
inline int xpass_rows_per_block(int rows, int mult) {
  int rpb = (mult == 1 || mult == 2 || mult == 4 ? mult : 2) * Line<N1>::LPI;
  while (rpb > Line<N1>::LPI && xpass_smem<R, N1>(rpb) > 96 * 1024) rpb /= 2;
  return rpb < rows ? rpb : rows;
}

// ---------------------------------------------------------------------------
// Batched complex GEMM of the restore pre-pass: block (bx, by, g) computes the
// 64 x 64 tile (by, bx) of product g.  256 threads, 4 x 4 outputs each; A and
// B are staged through shared memory in chunks of kGemmKC along K.
// ---------------------------------------------------------------------------
constexpr int kGemmT = 64, kGemmKC = 16;

template <typename R>
__global__ void __launch_bounds__(kThreads) cgemm_batched_kernel(const GemmDesc* __restrict__ descs) {
  using C = cx<R>;
  __shared__ C sA[kGemmT][kGemmKC + 1];
  __shared__ C sB[kGemmKC][kGemmT];
  const GemmDesc d = descs[blockIdx.z];
  const int m0 = blockIdx.y * kGemmT, n0 = blockIdx.x * kGemmT;
  if (m0 >= d.M || n0 >= d.N) return;
  const C* A = reinterpret_cast<const C*>(d.A);
  const C* B = reinterpret_cast<const C*>(d.B);
  C* Cm = reinterpret_cast<C*>(d.C);
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  C acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = czero<C>();
  for (int k0 = 0; k0 < d.K; k0 += kGemmKC) {
    for (int i = tid; i < kGemmT * kGemmKC; i += kThreads) {
      const int r = i / kGemmKC, k = i - r * kGemmKC;
      const int gm = m0 + r, gk = k0 + k;
      sA[r][k] = (gm < d.M && gk < d.K) ? A[(size_t)gm * d.K + gk] : czero<C>();
    }
    for (int i = tid; i < kGemmKC * kGemmT; i += kThreads) {
      const int k = i / kGemmT, c = i - k * kGemmT;
      const int gk = k0 + k, gn = n0 + c;
      sB[k][c] = (gk < d.K && gn < d.N) ? B[(size_t)gk * d.N + gn] : czero<C>();
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < kGemmKC; ++k) {
      C a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = sA[ty + 16 * i][k];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = sB[k][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) cfma(acc[i][j], a[i], b[j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < d.N) Cm[(size_t)gm * d.N + gn] = acc[i][j];
    }
  }
}

// ---------------------------------------------------------------------------
// The per-field work of a yz block (x, p), G fields per round: forward y DFT
// of rows z < Kz, z DFT x Hadamard with the slab x inverse z DFT of every
// column, inverse y DFT, corner written back in place.  `op` is the slab
// T~_p[x]: element (z, y) at op[y * op_cs + z * op_es] (shared memory [z][y]
// with an odd row pitch, or global memory [y][z] so that a team's z-line
// reads are contiguous); `planes` holds G planes of N3 / 2 rows of pitch
// N2 + 1 (a forward z line reads only its first half, an inverse one writes
// only rows z < Kz <= N3/2).  The G fields of a round share the phase
// barriers; each phase runs the unchanged line loop once per field.
// ---------------------------------------------------------------------------
template <typename R, int N2, int N3, int G, bool OP_GLOBAL>
__device__ __forceinline__ void yz_fields(const YZParams& P, int x, int p, cx<R>* planes, cx<R>* xs,
                                          const cx<R>* tw2, const cx<R>* tw3, const cx<R>* op,
                                          int op_cs, int op_es) {
  using C = cx<R>;
  constexpr int PY = N2 + 1;
  constexpr int PS = (N3 / 2) * PY;          // plane stride
  const int tid = threadIdx.x;
  const int Ky = P.Ky, Kz = P.Kz;
  __syncthreads();
  // rows Kz .. N3/2 - 1 stay zero for every field
  for (int g = 0; g < G; ++g)
    for (int i = tid; i < (N3 / 2 - Kz) * N2; i += kThreads) {
      const int z = Kz + i / N2, y = i % N2;
      planes[g * PS + z * PY + y] = czero<C>();
    }
  TeamPos<N2> ty;
  TeamPos<N3> tz;
  C* xy = ty.xs(xs);
  C* xz = tz.xs(xs);
  // a lane keeps its z-line position for every column and field: its
  // stage-1 twiddles W_N3^(t c) are computed once here (square z shapes);
  // with N2 = N3 the y-lines use the same team positions and twiddles
  constexpr bool kSqZ = Line<N3>::R1 == Line<N3>::R2;
  C wz[kSqZ ? Line<N3>::R1 : 1];
  if constexpr (kSqZ) twiddle_powers<Line<N3>::R1>(tw3[tz.t], wz);
  C* inter = reinterpret_cast<C*>(P.inter);
  const int hy = N2 / 2;
  const size_t fstride = (size_t)P.n1 * Kz * Ky;   // between consecutive fields
  // each thread owns up to kPre elements of a field's Kz x N2/2 input
  // corner; the next round's are loaded into registers during this one
  constexpr int kCorner = (N3 / 2) * (N2 / 2) / kThreads;
  constexpr int kPre = kCorner < 1 ? 1 : kCorner;
  constexpr bool kUsePre = kCorner * G <= 8;                                 // register budget
  const bool fits = kUsePre && Kz * hy <= kPre * kThreads;
  C pre[kUsePre ? G * kPre : 1];
  auto prefetch = [&](int j0) {
    if constexpr (kUsePre) {
      const C* io = inter + (((size_t)p * P.nf + j0) * P.n1 + x) * (size_t)(Kz * Ky);
#pragma unroll
      for (int g = 0; g < G; ++g)
#pragma unroll
        for (int k = 0; k < kPre; ++k) {
          const int i = tid + k * kThreads;
          const int z = i / hy, y = i - z * hy;
          pre[g * kPre + k] = (j0 + g < P.nf && i < Kz * hy && y < Ky) ? io[g * fstride + z * Ky + y] : czero<C>();
        }
    }
  };
  if (fits) prefetch(0);
  for (int j0 = 0; j0 < P.nf; j0 += G) {
    const int ng = min(G, P.nf - j0);
    C* io = inter + (((size_t)p * P.nf + j0) * P.n1 + x) * (size_t)(Kz * Ky);
    __syncthreads();
    if (fits) {
      if constexpr (kUsePre) {
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
          for (int k = 0; k < kPre; ++k) {
            const int i = tid + k * kThreads;
            const int z = i / hy, y = i - z * hy;
            if (g < ng && i < Kz * hy) planes[g * PS + z * PY + y] = pre[g * kPre + k];
          }
      }
      if (j0 + G < P.nf) prefetch(j0 + G);
    } else if constexpr (OP_GLOBAL) {
      // batches of kLd loads per thread in flight before their stores
      constexpr int kLd = 8;
      for (int g = 0; g < ng; ++g)
        for (int i0 = tid; i0 < Kz * hy; i0 += kLd * kThreads) {
          C v[kLd];
#pragma unroll
          for (int j = 0; j < kLd; ++j) {
            const int i = i0 + j * kThreads;
            const int z = i / hy, y = i - z * hy;
            v[j] = (i < Kz * hy && y < Ky) ? io[g * fstride + z * Ky + y] : czero<C>();
          }
#pragma unroll
          for (int j = 0; j < kLd; ++j) {
            const int i = i0 + j * kThreads;
            const int z = i / hy, y = i - z * hy;
            if (i < Kz * hy) planes[g * PS + z * PY + y] = v[j];
          }
        }
    } else {
      for (int g = 0; g < ng; ++g)
        for (int i = tid; i < Kz * hy; i += kThreads) {
          const int z = i / hy, y = i - z * hy;
          planes[g * PS + z * PY + y] = (y < Ky) ? io[g * fstride + z * Ky + y] : czero<C>();
        }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < ng; ++g) {
      C* plane = planes + g * PS;
      for (int base = 0; base < Kz; base += Line<N2>::LPI) {
        const int ln = base + ty.line;
        const bool act = ln < Kz;
        line_fft<N2, -1, true>(plane + (act ? ln : 0) * PY, 1, xy, tw2, ty.t, act, N2,
                               (kSqZ && N2 == N3) ? wz : nullptr);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < ng; ++g) {
      C* plane = planes + g * PS;
      for (int base = 0; base < N2; base += Line<N3>::LPI) {
        const int col = base + tz.line;
        const bool act = col < N2;
        const int cc = act ? col : 0;
        line_conv<N3, OP_GLOBAL>(plane + cc, PY, xz, tw3, op + (size_t)cc * op_cs, op_es, tz.t, act, Kz,
                                 kSqZ ? wz : nullptr);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int g = 0; g < ng; ++g) {
      C* plane = planes + g * PS;
      for (int base = 0; base < Kz; base += Line<N2>::LPI) {
        const int ln = base + ty.line;
        const bool act = ln < Kz;
        line_fft<N2, +1, false>(plane + (act ? ln : 0) * PY, 1, xy, tw2, ty.t, act, Ky,
                                (kSqZ && N2 == N3) ? wz : nullptr);
      }
    }
    __syncthreads();
    for (int g = 0; g < ng; ++g)
      for (int i = tid; i < Kz * Ky; i += kThreads) {
        const int z = i / Ky, y = i - z * Ky;
        io[g * fstride + i] = planes[g * PS + z * PY + y];
      }
  }
}

// ---------------------------------------------------------------------------
// The same batched products on the tensor cores (3xTF32, complex64): block
// (bx, by, g) computes the 64 x 64 output tile (by, bx) of product g with
// tc_cgemm64.  The launch asks for kTcGemmSmem bytes of shared memory so
// that at most four blocks share an SM and its 512 TMEM columns.
// ---------------------------------------------------------------------------
constexpr size_t kTcGemmSmem = 56 * 1024;
// contraction chunk of the CUDA-core TT-like slab restore (slab_tt_chunked)
constexpr int kRestoreKC = 64;
// Large-plane restore tiles: a contraction of at least kPipeMinK runs the
// pipelined tile (tc_cgemm64_pipe: chunks of 16 with the next chunk's copies
// and split overlapping the previous MMAs), a shorter one the single-buffer
// tile with chunks of kTcKCLarge, whose fewer round trips win there (64^3
// TT-4D, K = 541: yz 31.4 -> 29.0 ms pipelined; 64^3 H-Tucker, K <= 61:
// 9.5 -> 10.5 ms pipelined, so it keeps the long chunks)
constexpr int kPipeMinK = 128;
constexpr int kTcKCLarge = 32;

template <bool C_GLOBAL, bool BF16>
__device__ __forceinline__ void tc_cgemm64_strided(TcState& s, float2* ring, int M, int N, int K, const float2* A,
                                                   long long am, long long ak, const float2* B, long long bk,
                                                   long long bn, float2* C, int ldc, float scale) {
  if (K >= kPipeMinK) {
    tc_cgemm64_pipe<C_GLOBAL, BF16>(s, ring, M, N, K, A, am, ak, B, bk, bn, C, ldc, scale);
  } else {
    tc_cgemm64<C_GLOBAL, BF16, kTcKCLarge>(
        s, M, N, K, [&](int m, int k) { return A[m * am + k * ak]; },
        [&](int k, int n) { return B[k * bk + n * bn]; }, C, ldc, scale);
  }
}

template <bool BF16>   // BF16: BF16x3 products, else 3xTF32 (single TF32 with `single`)
__global__ void __launch_bounds__(kThreads) cgemm_batched_tc_kernel(const GemmDesc* __restrict__ descs,
                                                                    int* status, int single) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ uint64_t tc_bar;
  const GemmDesc d = descs[blockIdx.z];
  const int m0 = blockIdx.y * 64, n0 = blockIdx.x * 64;
  if (m0 >= d.M || n0 >= d.N) return;                     // uniform over the block
  const float2* A = reinterpret_cast<const float2*>(d.A) + (size_t)m0 * d.K;
  const float2* B = reinterpret_cast<const float2*>(d.B) + n0;
  float2* Cm = reinterpret_cast<float2*>(d.C) + (size_t)m0 * d.N + n0;
  const int K = d.K, N = d.N;
  TcState tc = tc_setup(smem_raw, &tc_bar, &tmem_slot);
  tc.single = single != 0;
  tc_cgemm64<true, BF16>(tc, min(64, d.M - m0), min(64, d.N - n0), K, [&](int m, int k) { return A[(size_t)m * K + k]; },
                   [&](int k, int n) { return B[(size_t)k * N + n]; }, Cm, N, 1.0f);
  if (!tc.ok && threadIdx.x == 0) atomicOr(status, kStatusTcTimeout);
  tc_teardown(tc);
}

// ---------------------------------------------------------------------------
// yz pass.  FMT 0: plain operator from global memory.  FMT 1: Tucker-like
// restore of the slab (Fig. 3(a) steps 2-3, with the factors of the format):
//   T~_p[x][y][z] = sum_{b,c} U2[y][b] H_p[x][b][c] U3[z][c]
// FMT 2: TT-like restore (Fig. 4(a) step 2, Fig. 4(b) step 3):
//   T~_p[x][y][z] = sum_b T1[x][y][b] R_p[z][b]
// ---------------------------------------------------------------------------
template <typename R, int N2, int N3>
struct YZLayout {
  static constexpr int PY = N2 + 1;
  static constexpr int XW = (Line<N2>::XW > Line<N3>::XW) ? Line<N2>::XW : Line<N3>::XW;
  static constexpr size_t fixed_elems = (size_t)N3 * PY + N2 + N3;   // Tt + twiddles
  static constexpr int G = 2;                                          // fields per round
  static constexpr size_t plane_elems = (size_t)G * (N3 / 2) * PY + kWarps * XW;
  // restore work space.  FMT 1: Gt (rb x N2) plus, before stage B, Ht
  // (rb x ra) and U2t (ra x N2), then U3 (N3 x rb).  FMT 2: one chunk of the
  // contraction over rb, T1[x] (kRestoreKC x (N2 + 1)) and U3 (N3 x kRestoreKC)
  static size_t restore_elems(int fmt, int ra, int rb) {
    if (fmt == 2) {
      const size_t kc = rb < kRestoreKC ? (size_t)rb : (size_t)kRestoreKC;
      return kc * (N2 + 1) + (size_t)N3 * kc;
    }
    const size_t a = (size_t)rb * ra + (size_t)ra * N2, b = (size_t)N3 * rb;
    return (size_t)rb * N2 + (a > b ? a : b);
  }
  // tensor-core restore: operand chunks + mbarrier, then G (rb x (N2 + 1), FMT 1)
  static size_t restore_bytes_tc(int fmt, int rb) {
    return kTcSmemBytes + (fmt == 1 ? sizeof(cx<R>) * (size_t)rb * (N2 + 1) : 0);
  }
  static size_t smem_bytes(int fmt, int ra, int rb, bool tc = false) {
    size_t work = sizeof(cx<R>) * plane_elems;
    if (fmt != 0) {
      const size_t r = tc ? restore_bytes_tc(fmt, rb) : sizeof(cx<R>) * restore_elems(fmt, ra, rb);
      if (r > work) work = r;
    }
    return sizeof(cx<R>) * fixed_elems + work;
  }
};

// Row tile of the CUDA-core slab products (N3 rows x N2 columns, 32 TN columns
// per warp item): as many rows as give every warp of the block an item.
template <int N2, int N3>
struct SlabTile {
  static constexpr int TN = N2 >= 64 ? 2 : 1;
  static constexpr int NCB = (N2 + 32 * TN - 1) / (32 * TN);
  static constexpr int TM0 = N3 * NCB / kWarps;
  static constexpr int TM = TM0 < 1 ? 1 : (TM0 > 8 ? 8 : TM0);
};

// TT-like slab on the CUDA cores, the contraction over rb in chunks of
// kRestoreKC staged in shared memory (any rb fits):
//   Tt[z * PY + y] = scale * sum_b U3[z * rb + b] H[y * rb + b]
// Every warp keeps its output tiles in registers across the chunks.
template <int N2, int N3, typename C>
__device__ __forceinline__ void slab_tt_chunked(int rb, const C* __restrict__ H, const C* __restrict__ U3,
                                                C* work, C* Tt, int PY, typename real_of<C>::type scale) {
  using T = SlabTile<N2, N3>;
  constexpr int TM = T::TM, TN = T::TN, NCB = T::NCB;
  constexpr int KC = kRestoreKC, GP = N2 + 1;
  constexpr int ITEMS = ((N3 + TM - 1) / TM) * NCB;
  constexpr int IPW = (ITEMS + kWarps - 1) / kWarps;
  const int kcap = rb < KC ? rb : KC;
  C* Gc = work;                  // chunk of T1[x]: Gc[b * GP + y] = H[y * rb + k0 + b]
  C* Uc = Gc + kcap * GP;        // chunk of U3:    Uc[z * kcap + b] = U3[z * rb + k0 + b]
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  C acc[IPW][TM][TN];
#pragma unroll
  for (int it = 0; it < IPW; ++it)
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[it][i][j] = czero<C>();
  for (int k0 = 0; k0 < rb; k0 += KC) {
    const int kc = rb - k0 < KC ? rb - k0 : KC;
    __syncthreads();                               // previous chunk consumed
    for (int i = tid; i < N2 * kc; i += kThreads) {
      const int y = i / kc, b = i - y * kc;
      Gc[b * GP + y] = H[(size_t)y * rb + k0 + b];
    }
    for (int i = tid; i < N3 * kc; i += kThreads) {
      const int z = i / kc, b = i - z * kc;
      Uc[z * kcap + b] = U3[(size_t)z * rb + k0 + b];
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < IPW; ++it) {
      const int item = w + it * kWarps;
      if (item >= ITEMS) break;
      const int m0 = (item / NCB) * TM, n0 = (item % NCB) * (32 * TN);
      for (int k = 0; k < kc; ++k) {
        C b[TN];
#pragma unroll
        for (int j = 0; j < TN; ++j) {
          const int n = n0 + lane + 32 * j;
          b[j] = n < N2 ? Gc[k * GP + n] : czero<C>();
        }
#pragma unroll
        for (int i = 0; i < TM; ++i) {
          const int m = m0 + i;
          const C a = m < N3 ? Uc[m * kcap + k] : czero<C>();
#pragma unroll
          for (int j = 0; j < TN; ++j) cfma(acc[it][i][j], a, b[j]);
        }
      }
    }
  }
#pragma unroll
  for (int it = 0; it < IPW; ++it) {
    const int item = w + it * kWarps;
    if (item >= ITEMS) break;
    const int m0 = (item / NCB) * TM, n0 = (item % NCB) * (32 * TN);
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + i;
      if (m >= N3) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + lane + 32 * j;
        if (n < N2) Tt[m * PY + n] = mk<C>(acc[it][i][j].x * scale, acc[it][i][j].y * scale);
      }
    }
  }
}

// Item (x, p) of the fused yz pass, by the whole block: the slab of direction
// p at x loaded or restored into shared memory, then every field of p.
// `smem_raw` holds YZLayout::smem_bytes; `tcp` is the block's tensor-core
// state (TC != 0, set up by the caller, whose operand staging this item
// points at its own work area).
template <typename R, int N2, int N3, int FMT, int TC>   // TC: 0 CUDA cores, 1 3xTF32, 2 BF16x3
__device__ __forceinline__ void yz_body(const YZParams& P, int x, int p, unsigned char* smem_raw, TcState* tcp) {
  using C = cx<R>;
  using LY = YZLayout<R, N2, N3>;
  constexpr int PY = LY::PY;
  C* Tt = reinterpret_cast<C*>(smem_raw);   // N3 x PY, operator slab [z][y]
  C* tw2 = Tt + N3 * PY;
  C* tw3 = tw2 + N2;
  C* work = tw3 + N3;
  C* plane = work;                          // LY::G planes of N3/2 x PY, field [z][y]
  C* xs = plane + LY::G * (N3 / 2) * PY;
  const int tid = threadIdx.x;
  for (int i = tid; i < N2; i += kThreads) tw2[i] = reinterpret_cast<const C*>(P.tw2)[i];
  for (int i = tid; i < N3; i += kThreads) tw3[i] = reinterpret_cast<const C*>(P.tw3)[i];

  if constexpr (FMT == 0) {
    const C* op = reinterpret_cast<const C*>(P.op) + ((size_t)p * P.n1 + x) * (N3 * N2);
    for (int i = tid; i < N3 * N2; i += kThreads) {
      const int z = i / N2, y = i - z * N2;
      Tt[z * PY + y] = op[i];
    }
  } else {
    const SlabDesc d = P.desc[p];
    const int ra = d.ra, rb = d.rb;
    if (ra > P.rmax_a || rb > P.rmax_b) {
      if (tid == 0) atomicOr(P.status, kStatusRankOverflow);
      return;
    }
    const C* H = reinterpret_cast<const C*>(d.h) + (size_t)x * d.hx;
    if constexpr (TC != 0) {
      // tensor cores, 3xTF32 or BF16x3 (tc_cgemm.cuh); factors read straight from L2
      TcState& tc = *tcp;
      tc.buf = reinterpret_cast<float*>(work);
      const float2* U3 = reinterpret_cast<const float2*>(d.u3);
      const float2* Hf = reinterpret_cast<const float2*>(H);
      if constexpr (FMT == 1) {
        float2* G = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(work) + kTcSmemBytes);
        const float2* U2 = reinterpret_cast<const float2*>(d.u2);
        // G[c][y] = sum_b H_p[x][b][c] U2[y][b]; odd pitch PY: the epilogue
        // writes one row per lane
        tc_cgemm64<false, TC == 2>(tc, rb, N2, ra, [&](int c, int b) { return Hf[b * rb + c]; },
                   [&](int b, int y) { return U2[y * ra + b]; }, G, PY, 1.0f);
        // slab[z][y] = scale sum_c U3[z][c] G[c][y]
        tc_cgemm64<false, TC == 2>(tc, N3, N2, rb, [&](int z, int c) { return U3[z * rb + c]; },
                   [&](int c, int y) { return G[c * PY + y]; }, reinterpret_cast<float2*>(Tt), PY,
                   (float)P.scale);
      } else {
        // slab[z][y] = scale sum_b R_p[z][b] T1[x][y][b]
        tc_cgemm64<false, TC == 2>(tc, N3, N2, rb, [&](int z, int b) { return U3[z * rb + b]; },
                   [&](int b, int y) { return Hf[y * rb + b]; }, reinterpret_cast<float2*>(Tt), PY,
                   (float)P.scale);
      }
    } else {
      // CUDA cores; row tiles sized so that every warp has an output tile
      using ST = SlabTile<N2, N3>;
      const C* U3 = reinterpret_cast<const C*>(d.u3);
      if constexpr (FMT == 1) {
        C* Gt = work;                            // rb x N2
        C* U3s = Gt + rb * N2;                   // N3 x rb (stage B)
        C* Ht = Gt + rb * N2;                    // rb x ra
        C* U2t = Ht + rb * ra;                   // ra x N2
        const C* U2 = reinterpret_cast<const C*>(d.u2);
        for (int i = tid; i < ra * rb; i += kThreads) {
          const int b = i / rb, c = i - b * rb;
          Ht[c * ra + b] = H[i];
        }
        for (int i = tid; i < N2 * ra; i += kThreads) {
          const int y = i / ra, b = i - y * ra;
          U2t[b * N2 + y] = U2[i];
        }
        __syncthreads();
        block_cgemm<(N2 >= 64 ? 8 : 4), ST::TN>(rb, N2, ra, Ht, ra, U2t, N2, Gt, N2, (R)1);
        __syncthreads();
        for (int i = tid; i < N3 * rb; i += kThreads) U3s[i] = U3[i];
        __syncthreads();
        block_cgemm<ST::TM, ST::TN>(N3, N2, rb, U3s, rb, Gt, N2, Tt, PY, (R)P.scale);
      } else {
        slab_tt_chunked<N2, N3>(rb, H, U3, work, Tt, PY, (R)P.scale);
      }
    }
  }
  yz_fields<R, N2, N3, LY::G, false>(P, x, p, plane, xs, tw2, tw3, Tt, 1, PY);
}

// One (x, p) item per block, or (inst != null) the batch mode over
// the items (instance, x, p), p-major, of instances of this shape class.
template <typename R, int N2, int N3, int FMT, int TC>   // TC: 0 CUDA cores, 1 3xTF32, 2 BF16x3
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) yz_kernel(YZParams P, const BatchYZ* __restrict__ inst, int ninst,
                                                         long long total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ uint32_t tmem_slot;
  __shared__ uint64_t tc_bar;
  TcState tc;
  if constexpr (FMT != 0 && TC != 0) tc = tc_setup(smem_raw, &tc_bar, &tmem_slot);
  // one code path for both modes; the item's parameters in registers (a
  // shared copy would be re-read after every shared-memory store)
  // a block's items advance by gridDim.x: the instance is looked up only
  // when an item leaves the current instance's range
  const long long count = inst ? total : 1;
  long long lo = 1, hi = 0;
  YZParams sp = P;
  for (long long item = inst ? blockIdx.x : 0; item < count; item += gridDim.x) {
    if (inst && (item < lo || item >= hi)) {
      const int i = find_instance(inst, ninst, item);
      lo = inst[i].item0;
      hi = i + 1 < ninst ? inst[i + 1].item0 : total;
      sp = inst[i].P;
    }
    if (inst) __syncthreads();                       // the previous item is done with shared memory
    const int local = inst ? (int)(item - lo) : 0;
    const int x = inst ? local % sp.n1 : (int)blockIdx.x;
    const int p = inst ? local / sp.n1 : sp.p0 + (int)blockIdx.y;
    if constexpr (FMT != 0 && TC != 0) tc.single = sp.tc_single != 0;
    const bool ok_before = tc.ok;
    yz_body<R, N2, N3, FMT, TC>(sp, x, p, smem_raw, &tc);
    if constexpr (FMT != 0 && TC != 0) {
      // a wait that ran out marks the plan of the item it happened in
      if (ok_before && !tc.ok && threadIdx.x == 0) atomicOr(sp.status, kStatusTcTimeout);
    }
  }
  if constexpr (FMT != 0 && TC != 0) tc_teardown(tc);
}

// ---------------------------------------------------------------------------
// yz pass for y-z planes too large for the slab and the field plane to share
// the shared memory (n2 x n3 = 128 x 128, 256 x 64, 256 x 128).  Persistent
// blocks walk the (x, p) items; the slab T~_p[x] stays in global memory: the
// plain operator in place, a restored slab in the block's own scratch slot,
// which stays resident in L2 while the block's fields use it.  Both are
// stored column by column ([y][z], z fastest), so that the eight lanes of a
// z-line team read consecutive elements.  Shared memory holds the twiddles,
// half a field plane and the exchange buffers; the restore's staging
// (tensor-core operand chunks) reuses the plane.  Two FP32 blocks share an
// SM (the launch bound caps their registers at 128).
// ---------------------------------------------------------------------------
template <typename R, int N2, int N3>
struct YZLLayout {
  static constexpr int PY = N2 + 1;
  static constexpr int XW = (Line<N2>::XW > Line<N3>::XW) ? Line<N2>::XW : Line<N3>::XW;
  static constexpr size_t plane_elems = (size_t)(N3 / 2) * PY + kWarps * XW;
  static size_t smem_bytes(int fmt, bool tc) {
    size_t work = sizeof(cx<R>) * plane_elems;
    // tensor-core restore: two staging buffers and the operand ring of the
    // pipelined tile, or the single-buffer tile's long chunks
    constexpr size_t kPipe = tc_pipe_staging_bytes<false>() + kPipeRingBytes;
    constexpr size_t kStage = tc_smem_bytes<kTcKCLarge>();
    constexpr size_t kTcWork = kPipe > kStage ? kPipe : kStage;
    if (fmt != 0 && tc && kTcWork > work) work = kTcWork;
    return sizeof(cx<R>) * (N2 + N3) + work;
  }
  // global scratch per block: the slab, then G (rb x N2) of the Tucker-like
  // restore
  static long long slot_elems(int fmt, int rb) {   // slab [y][z], then G
    return fmt == 0 ? 0 : (long long)N3 * N2 + (fmt == 1 ? (long long)rb * N2 : 0);
  }
};

template <typename R, int N2, int N3, int FMT, int TC>   // TC: 0 CUDA cores, 1 3xTF32, 2 BF16x3
__global__ void __launch_bounds__(kThreads, sizeof(R) == 4 ? 2 : 1) yzl_kernel(YZParams P) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw2 = reinterpret_cast<C*>(smem_raw);
  C* tw3 = tw2 + N2;
  C* plane = tw3 + N3;                      // N3/2 x (N2 + 1), then exchange
  C* xs = plane + (N3 / 2) * (N2 + 1);
  const int tid = threadIdx.x;
  for (int i = tid; i < N2; i += kThreads) tw2[i] = reinterpret_cast<const C*>(P.tw2)[i];
  for (int i = tid; i < N3; i += kThreads) tw3[i] = reinterpret_cast<const C*>(P.tw3)[i];
  C* slot = nullptr;
  C* G = nullptr;
  if constexpr (FMT != 0) {
    slot = reinterpret_cast<C*>(P.slab_scratch) + (size_t)blockIdx.x * P.slot_elems;
    G = slot + (size_t)N3 * N2;
  }
  __shared__ uint32_t tmem_slot;
  __shared__ uint64_t tc_bar[2];
  TcState tc;
  if constexpr (TC != 0) {
    tc = tc_setup(plane, &tc_bar[0], &tmem_slot, &tc_bar[1]);
    tc.single = P.tc_single != 0;
  }
  const int items = P.n1 * P.n_dir;
  for (int it = blockIdx.x; it < items; it += gridDim.x) {
    const int x = it % P.n1, p = P.p0 + it / P.n1;
    const C* op;   // [y][z]
    if constexpr (FMT == 0) {
      op = reinterpret_cast<const C*>(P.op) + ((size_t)p * P.n1 + x) * (N3 * N2);
    } else {
      const SlabDesc d = P.desc[p];
      const int ra = d.ra, rb = d.rb;
      const bool bad = ra > P.rmax_a || rb > P.rmax_b || (TC != 0 && FMT == 1 && rb > 64);
      if (bad) {
        if (tid == 0) atomicOr(P.status, kStatusRankOverflow);
        continue;                                  // uniform over the block
      }
      const C* H = reinterpret_cast<const C*>(d.h) + (size_t)x * d.hx;
      const C* U2 = reinterpret_cast<const C*>(d.u2);
      const C* U3 = reinterpret_cast<const C*>(d.u3);
      __syncthreads();                             // previous item done with slot and plane
      if constexpr (TC != 0) {
        const float2* Hf = reinterpret_cast<const float2*>(H);
        const float2* U2f = reinterpret_cast<const float2*>(U2);
        const float2* U3f = reinterpret_cast<const float2*>(U3);
        float2* Gf = reinterpret_cast<float2*>(G);
        float2* Sf = reinterpret_cast<float2*>(slot);
        // slab[y][z] tiles of 64 x 64 on the tensor cores; the staging buffers
        // (and the pipelined tile's operand ring) take the plane's space
        constexpr bool kBf = TC == 2;
        float2* ring = reinterpret_cast<float2*>(reinterpret_cast<unsigned char*>(plane) +
                                                 tc_pipe_staging_bytes<kBf>());
        if constexpr (FMT == 1) {
          // G[c][y] = sum_b H_p[x][b][c] U2[y][b]; slab[y][z] = scale sum_c G[c][y] U3[z][c]
          for (int y0 = 0; y0 < N2; y0 += 64)
            tc_cgemm64_strided<true, kBf>(tc, ring, rb, 64, ra, Hf, 1, rb, U2f + (size_t)y0 * ra, 1, ra, Gf + y0, N2,
                                       1.0f);
          for (int y0 = 0; y0 < N2; y0 += 64)
            for (int z0 = 0; z0 < N3; z0 += 64)
              tc_cgemm64_strided<true, kBf>(tc, ring, 64, 64, rb, Gf + y0, 1, N2, U3f + (size_t)z0 * rb, 1, rb,
                                         Sf + (size_t)y0 * N3 + z0, N3, (float)P.scale);
        } else {
          // slab[y][z] = scale sum_b T1[x][y][b] R_p[z][b]
          for (int y0 = 0; y0 < N2; y0 += 64)
            for (int z0 = 0; z0 < N3; z0 += 64)
              tc_cgemm64_strided<true, kBf>(tc, ring, 64, 64, rb, Hf + (size_t)y0 * rb, rb, 1, U3f + (size_t)z0 * rb,
                                         1, rb, Sf + (size_t)y0 * N3 + z0, N3, (float)P.scale);
        }
      } else {
        if constexpr (FMT == 1) {
          // G[c][y] = sum_b H[x][b][c] U2[y][b]
          block_cgemm_strided(rb, N2, ra, H, 1, rb, U2, 1, ra, G, N2, (R)1);
          __syncthreads();
          // slab[y][z] = scale sum_c G[c][y] U3[z][c]
          block_cgemm_strided(N2, N3, rb, G, 1, N2, U3, 1, rb, slot, N3, (R)P.scale);
        } else {
          // slab[y][z] = scale sum_b T1[x][y][b] R_p[z][b]
          block_cgemm_strided(N2, N3, rb, H, rb, 1, U3, 1, rb, slot, N3, (R)P.scale);
        }
      }
      __syncthreads();
      op = slot;
    }
    yz_fields<R, N2, N3, 1, true>(P, x, p, plane, xs, tw2, tw3, op, N3, 1);
  }
  if constexpr (TC != 0) {
    if (!tc.ok && tid == 0) atomicOr(P.status, kStatusTcTimeout);
    tc_teardown(tc);
  }
}

}  // namespace fmm
