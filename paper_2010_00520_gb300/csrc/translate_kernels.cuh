// Kernels of the translation stage (Eq. 5) and of the Tucker-3D restoration
// (Sec. II.C, Fig. 3(a)).
//
// A field A (Kz x Ky x Kx, x fastest) is translated in three passes:
//   xfwd  : rows r = z Ky + y: zero-pad x to n1, forward DFT along x, write
//           the x-spectrum transposed to the intermediate I[f][x][r]
//   yz    : one block per (x, direction p): the operator slab T~_p[x][:][:]
//           is loaded (format NONE) or restored (Tucker-3D) into shared
//           memory once, then for every field of direction p: forward DFT
//           along y (rows z < Kz), along z (columns) fused with the Hadamard
//           product and the inverse DFT along z, inverse DFT along y, and the
//           Kz x Ky corner is written back in place
//   xinv  : inverse DFT along x of every row, first Kx entries written out
// The 1 / (n1 n2 n3) of the inverse transform is folded into the operator.
#pragma once

#include "fft_core.cuh"
#include "plan_internal.h"

namespace fmm {

// Status-word bits set by kernels instead of faulting.
enum : int {
  kStatusRankOverflow = 1,   // a direction's ranks exceed the launch's shared memory
  kStatusBadShape = 2,       // launch shape does not match the problem
};

struct XPassParams {
  const void* src;   // xfwd: S_in; xinv: intermediate
  void* dst;         // xfwd: intermediate; xinv: S_out
  const void* tw;    // W_n1^m table
  int Kx, rows;      // rows = Ky * Kz per field
  int rows_per_block;
};

struct YZParams {
  void* inter;       // [F][n1][Kz][Ky]
  const void* tw2, *tw3;
  int Ky, Kz, n1, nf;  // nf = fields per direction (2 nrhs)
  const void* op;      // plain: [p][x][z][y], scaled
  const Tucker3DDesc* desc;
  const void* pack;
  const void* hbuf;
  double scale;        // restore scale 1 / (n1 n2 n3)
  int rmax2, rmax3;    // shared-memory capacity of the launch (ranks)
  int* status;
  int variant;         // yz launch variant (FMMFFT_KEY_YZ_VARIANT)
};

struct HParams {
  const Tucker3DDesc* desc;
  const void* pack;
  void* hbuf;
  int n1;
  int cols_per_block;
  int rmax1;
  int* status;
};

// ---------------------------------------------------------------------------
// x passes
// ---------------------------------------------------------------------------
template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xfwd_kernel(XPassParams P) {
  using C = cx<R>;
  using L = Line<N1>;
  constexpr int PX = N1 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xs = tw + N1;
  C* Q = xs + kWarps * L::XW;
  const int nrb = (P.rows + P.rows_per_block - 1) / P.rows_per_block;
  const int f = blockIdx.x / nrb;
  const int r0 = (blockIdx.x - f * nrb) * P.rows_per_block;
  const int nr = min(P.rows_per_block, P.rows - r0);
  const C* src = reinterpret_cast<const C*>(P.src) + ((size_t)f * P.rows + r0) * P.Kx;
  C* dst = reinterpret_cast<C*>(P.dst);
  for (int i = threadIdx.x; i < N1; i += kThreads) tw[i] = reinterpret_cast<const C*>(P.tw)[i];
  const int half = N1 / 2;
  for (int i = threadIdx.x; i < nr * half; i += kThreads) {
    const int r = i / half, x = i - r * half;
    Q[r * PX + x] = (x < P.Kx) ? src[(size_t)r * P.Kx + x] : czero<C>();
  }
  __syncthreads();
  TeamPos<N1> tp;
  C* xt = tp.xs(xs);
  for (int base = 0; base < nr; base += L::LPI) {
    const int line = base + tp.line;
    const bool act = line < nr;
    line_fft<N1, -1, true>(Q + (act ? line : 0) * PX, 1, xt, tw, tp.t, act, N1);
  }
  __syncthreads();
  // I[f][x][r]: rows contiguous for fixed x
  for (int i = threadIdx.x; i < N1 * nr; i += kThreads) {
    const int x = i / nr, r = i - x * nr;
    dst[((size_t)f * N1 + x) * P.rows + r0 + r] = Q[r * PX + x];
  }
}

template <typename R, int N1>
__global__ void __launch_bounds__(kThreads) xinv_kernel(XPassParams P) {
  using C = cx<R>;
  using L = Line<N1>;
  constexpr int PX = N1 + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* xs = tw + N1;
  C* Q = xs + kWarps * L::XW;
  const int nrb = (P.rows + P.rows_per_block - 1) / P.rows_per_block;
  const int f = blockIdx.x / nrb;
  const int r0 = (blockIdx.x - f * nrb) * P.rows_per_block;
  const int nr = min(P.rows_per_block, P.rows - r0);
  const C* src = reinterpret_cast<const C*>(P.src);
  C* dst = reinterpret_cast<C*>(P.dst) + ((size_t)f * P.rows + r0) * P.Kx;
  for (int i = threadIdx.x; i < N1; i += kThreads) tw[i] = reinterpret_cast<const C*>(P.tw)[i];
  for (int i = threadIdx.x; i < N1 * nr; i += kThreads) {
    const int x = i / nr, r = i - x * nr;
    Q[r * PX + x] = src[((size_t)f * N1 + x) * P.rows + r0 + r];
  }
  __syncthreads();
  TeamPos<N1> tp;
  C* xt = tp.xs(xs);
  for (int base = 0; base < nr; base += L::LPI) {
    const int line = base + tp.line;
    const bool act = line < nr;
    line_fft<N1, +1, false>(Q + (act ? line : 0) * PX, 1, xt, tw, tp.t, act, P.Kx);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nr * P.Kx; i += kThreads) {
    const int r = i / P.Kx, x = i - r * P.Kx;
    dst[(size_t)r * P.Kx + x] = Q[r * PX + x];
  }
}

// Shared memory of the x passes (bytes).
template <typename R, int N1>
constexpr size_t xpass_smem(int rows_per_block) {
  return sizeof(cx<R>) * (N1 + kWarps * Line<N1>::XW + (size_t)rows_per_block * (N1 + 1));
}

// ---------------------------------------------------------------------------
// Tucker-3D restore, step 1 (Fig. 3(a)): H_p = U1_p . mat(C_p), an
// n1 x (r2 r3) matrix per direction; one block per (column chunk, p).
// ---------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(kThreads) tucker3d_h_kernel(HParams P) {
  using C = cx<R>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Tucker3DDesc d = P.desc[blockIdx.y];
  const int ncol = d.r2 * d.r3;
  const int c0 = blockIdx.x * P.cols_per_block;
  if (c0 >= ncol) return;
  if (d.r1 > P.rmax1) {
    if (threadIdx.x == 0) atomicOr(P.status, kStatusRankOverflow);
    return;
  }
  const int nc = min(P.cols_per_block, ncol - c0);
  C* sU1 = reinterpret_cast<C*>(smem_raw);          // n1 x r1
  C* sC = sU1 + P.n1 * d.r1;                         // r1 x cols_per_block
  const C* pack = reinterpret_cast<const C*>(P.pack);
  for (int i = threadIdx.x; i < P.n1 * d.r1; i += kThreads) sU1[i] = pack[d.off_u1 + i];
  for (int i = threadIdx.x; i < d.r1 * nc; i += kThreads) {
    const int a = i / nc, c = i - a * nc;
    sC[a * P.cols_per_block + c] = pack[d.off_core + (int64_t)a * ncol + c0 + c];
  }
  __syncthreads();
  C* H = reinterpret_cast<C*>(P.hbuf) + d.off_h + c0;
  block_cgemm<8, 2>(P.n1, nc, d.r1, sU1, d.r1, sC, P.cols_per_block, H, ncol, (R)1);
}

// ---------------------------------------------------------------------------
// yz pass.  FMT 0: plain operator from global memory.  FMT 1: Tucker-3D
// restore of the slab from H_p[x] (r2 x r3), U2_p and U3_p (Fig. 3(a),
// steps 2-3):  T~_p[x][y][z] = sum_{b,c} U2_p[y][b] H_p[x][b][c] U3_p[z][c].
// ---------------------------------------------------------------------------
template <typename R, int N2, int N3>
struct YZLayout {
  static constexpr int PY = N2 + 1;
  static constexpr int XW = (Line<N2>::XW > Line<N3>::XW) ? Line<N2>::XW : Line<N3>::XW;
  static constexpr size_t fixed_elems = (size_t)N3 * PY + N2 + N3;   // Tt + twiddles
  static constexpr size_t plane_elems = (size_t)N3 * PY + kWarps * XW;
  static size_t restore_elems(int r2, int r3) {
    const size_t a = (size_t)r3 * r2 + (size_t)r2 * N2, b = (size_t)N3 * r3;
    return (size_t)r3 * N2 + (a > b ? a : b);
  }
  static size_t smem_bytes(int fmt, int r2, int r3) {
    size_t work = plane_elems;
    if (fmt == 1) { const size_t r = restore_elems(r2, r3); if (r > work) work = r; }
    return sizeof(cx<R>) * (fixed_elems + work);
  }
};

template <typename R, int N2, int N3, int FMT>
__global__ void __launch_bounds__(kThreads, 1) yz_kernel(YZParams P) {
  using C = cx<R>;
  using LY = YZLayout<R, N2, N3>;
  constexpr int PY = LY::PY;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Tt = reinterpret_cast<C*>(smem_raw);   // N3 x PY, operator slab [z][y]
  C* tw2 = Tt + N3 * PY;
  C* tw3 = tw2 + N2;
  C* work = tw3 + N3;
  C* plane = work;                          // N3 x PY, field [z][y]
  C* xs = plane + N3 * PY;
  const int x = blockIdx.x, p = blockIdx.y;
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
    const Tucker3DDesc d = P.desc[p];
    const int r2 = d.r2, r3 = d.r3;
    if (r2 > P.rmax2 || r3 > P.rmax3) {
      if (tid == 0) atomicOr(P.status, kStatusRankOverflow);
      return;
    }
    const C* pack = reinterpret_cast<const C*>(P.pack);
    const C* H = reinterpret_cast<const C*>(P.hbuf) + d.off_h + (size_t)x * r2 * r3;
    C* Gt = work;                              // r3 x N2
    C* Ht = Gt + r3 * N2;                      // r3 x r2
    C* U2t = Ht + r3 * r2;                     // r2 x N2
    C* U3s = Ht;                               // N3 x r3 (after Gt is formed)
    for (int i = tid; i < r2 * r3; i += kThreads) {
      const int b = i / r3, c = i - b * r3;
      Ht[c * r2 + b] = H[i];
    }
    for (int i = tid; i < N2 * r2; i += kThreads) {
      const int y = i / r2, b = i - y * r2;
      U2t[b * N2 + y] = pack[d.off_u2 + i];
    }
    __syncthreads();
    block_cgemm<8, (N2 >= 64 ? 2 : 1)>(r3, N2, r2, Ht, r2, U2t, N2, Gt, N2, (R)1);
    __syncthreads();
    for (int i = tid; i < N3 * r3; i += kThreads) U3s[i] = pack[d.off_u3 + i];
    __syncthreads();
    block_cgemm<8, (N2 >= 64 ? 2 : 1)>(N3, N2, r3, U3s, r3, Gt, N2, Tt, PY, (R)P.scale);
  }
  __syncthreads();

  const int Ky = P.Ky, Kz = P.Kz;
  // rows Kz .. N3/2 - 1 stay zero for every field
  for (int i = tid; i < (N3 / 2 - Kz) * N2; i += kThreads) {
    const int z = Kz + i / N2, y = i % N2;
    plane[z * PY + y] = czero<C>();
  }
  TeamPos<N2> ty;
  TeamPos<N3> tz;
  C* xy = ty.xs(xs);
  C* xz = tz.xs(xs);
  C* inter = reinterpret_cast<C*>(P.inter);
  const int hy = N2 / 2;
  for (int j = 0; j < P.nf; ++j) {
    const size_t f = (size_t)p * P.nf + j;
    C* io = inter + (f * P.n1 + x) * (size_t)(Kz * Ky);
    __syncthreads();
    for (int i = tid; i < Kz * hy; i += kThreads) {
      const int z = i / hy, y = i - z * hy;
      plane[z * PY + y] = (y < Ky) ? io[z * Ky + y] : czero<C>();
    }
    __syncthreads();
    for (int base = 0; base < Kz; base += Line<N2>::LPI) {
      const int ln = base + ty.line;
      const bool act = ln < Kz;
      line_fft<N2, -1, true>(plane + (act ? ln : 0) * PY, 1, xy, tw2, ty.t, act, N2);
    }
    __syncthreads();
    for (int base = 0; base < N2; base += Line<N3>::LPI) {
      const int col = base + tz.line;
      const bool act = col < N2;
      const int cc = act ? col : 0;
      line_conv<N3>(plane + cc, PY, xz, tw3, Tt + cc, PY, tz.t, act, Kz);
    }
    __syncthreads();
    for (int base = 0; base < Kz; base += Line<N2>::LPI) {
      const int ln = base + ty.line;
      const bool act = ln < Kz;
      line_fft<N2, +1, false>(plane + (act ? ln : 0) * PY, 1, xy, tw2, ty.t, act, Ky);
    }
    __syncthreads();
    for (int i = tid; i < Kz * Ky; i += kThreads) {
      const int z = i / Ky, y = i - z * Ky;
      io[i] = plane[z * PY + y];
    }
  }
}

// ---------------------------------------------------------------------------
// yz pass, lane-split version (n2, n3 <= 64).  Every line transform runs in
// registers (one or two lanes per line, see Split<N>); shared memory holds the
// operator slab Tt[z][y] and G field planes [z][y] (pitch n2 + 1), so the y,
// z, Hadamard and inverse steps of G fields of direction p run per group of
// five barriers.  Inputs of a forward line beyond its K entries are never
// read, so no zero padding is stored.
// ---------------------------------------------------------------------------
template <typename R, int N2, int N3, int NT>
struct YZ2Layout {
  static constexpr int L2 = Split<N2>::L, L3 = Split<N3>::L;
  static constexpr int G = (NT / (N2 * L3)) > 0 ? (NT / (N2 * L3)) : 1;  // planes
  static constexpr int PP = N2 + 1;    // plane pitch
  // slab pitch: with two lanes per z-line, lanes l = 0, 1 read slab rows 2m
  // and 2m + 1 of the same column; a pitch of 8 (mod 16) complex elements puts
  // them in different bank pairs
  static constexpr int PT = (L3 == 2 && N2 % 16 == 0) ? N2 + 8 : N2;
  static constexpr size_t slab_elems = (size_t)N3 * PT;
  static constexpr size_t planes_elems = (size_t)G * N3 * PP;
  static size_t restore_elems(int r2, int r3) {
    const size_t r2p = (size_t)(r2 | 1);
    const size_t a = (size_t)r3 * r2p + (size_t)r2 * (N2 + 1), b = (size_t)N3 * r3;
    return (size_t)r3 * N2 + (a > b ? a : b);
  }
  static size_t smem_bytes(int fmt, int r2, int r3) {
    size_t work = planes_elems;
    if (fmt == 1) { const size_t r = restore_elems(r2, r3); if (r > work) work = r; }
    return sizeof(cx<R>) * (slab_elems + work);
  }
};

// Tucker-3D slab restore (Fig. 3(a) steps 2-3) into Tt[z * pt + y], scaled.
template <typename R, int N2, int N3, int NT>
__device__ __forceinline__ void restore_slab_tucker3d(const YZParams& P, int p, int x, cx<R>* Tt, int pt,
                                                      cx<R>* work) {
  using C = cx<R>;
  const Tucker3DDesc d = P.desc[p];
  const int r2 = d.r2, r3 = d.r3, r2p = d.r2 | 1;
  const int tid = threadIdx.x;
  const C* pack = reinterpret_cast<const C*>(P.pack);
  const C* H = reinterpret_cast<const C*>(P.hbuf) + d.off_h + (size_t)x * r2 * r3;
  C* Gt = work;                              // r3 x N2
  C* Ht = Gt + r3 * N2;                      // r3 x r2p   (Ht[c][b] = H[b][c])
  C* U2t = Ht + r3 * r2p;                    // r2 x (N2+1) (U2t[b][y] = U2[y][b])
  C* U3s = Ht;                               // N3 x r3 once Gt is formed
  for (int i = tid; i < r2 * r3; i += NT) {
    const int b = i / r3, c = i - b * r3;
    Ht[c * r2p + b] = H[i];
  }
  for (int i = tid; i < N2 * r2; i += NT) {
    const int y = i / r2, b = i - y * r2;
    U2t[b * (N2 + 1) + y] = pack[d.off_u2 + i];
  }
  __syncthreads();
  block_cgemm<8, (N2 >= 64 ? 2 : 1), C, NT / 32>(r3, N2, r2, Ht, r2p, U2t, N2 + 1, Gt, N2, (R)1);
  __syncthreads();
  for (int i = tid; i < N3 * r3; i += NT) U3s[i] = pack[d.off_u3 + i];
  __syncthreads();
  block_cgemm<8, (N2 >= 64 ? 2 : 1), C, NT / 32>(N3, N2, r3, U3s, r3, Gt, N2, Tt, pt, (R)P.scale);
}

template <typename R, int N2, int N3, int FMT, int NT>
__global__ void __launch_bounds__(NT) yz2_kernel(YZParams P) {
  using C = cx<R>;
  using LY = YZ2Layout<R, N2, N3, NT>;
  constexpr int L2 = LY::L2, L3 = LY::L3, G = LY::G, PP = LY::PP, PT = LY::PT;
  constexpr int M2 = Split<N2>::M, M3 = Split<N3>::M;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* Tt = reinterpret_cast<C*>(smem_raw);       // N3 x PT
  C* planes = Tt + LY::slab_elems;              // G x N3 x PP
  const int x = blockIdx.x, p = blockIdx.y;
  const int tid = threadIdx.x;

  if constexpr (FMT == 0) {
    const C* op = reinterpret_cast<const C*>(P.op) + ((size_t)p * P.n1 + x) * (N3 * N2);
    for (int i = tid; i < N3 * N2; i += NT) {
      const int z = i / N2, y = i - z * N2;
      Tt[z * PT + y] = op[i];
    }
  } else {
    const Tucker3DDesc d = P.desc[p];
    if (d.r2 > P.rmax2 || d.r3 > P.rmax3) {
      if (tid == 0) atomicOr(P.status, kStatusRankOverflow);
      return;
    }
    restore_slab_tucker3d<R, N2, N3, NT>(P, p, x, Tt, PT, planes);
  }

  const int Ky = P.Ky, Kz = P.Kz;
  const int fsz = Kz * Ky;
  C* inter = reinterpret_cast<C*>(P.inter);
#pragma unroll 1
  for (int g0 = 0; g0 < P.nf; g0 += G) {
    const int ng = min(G, P.nf - g0);
    __syncthreads();
    // fields g0 .. g0 + ng - 1 into planes rows z < Kz, columns y < Ky
    for (int i = tid; i < ng * fsz; i += NT) {
      const int j = i / fsz, r = i - j * fsz;
      const int z = r / Ky, y = r - z * Ky;
      const size_t f = (size_t)p * P.nf + g0 + j;
      planes[(j * N3 + z) * PP + y] = inter[(f * P.n1 + x) * fsz + r];
    }
    __syncthreads();
    // forward y: rows (j, z < Kz); inputs y < Ky, all n2 outputs
    {
      const int l = tid % L2;
#pragma unroll 1
      for (int base = 0; base < ng * Kz; base += NT / L2) {
        const int li = base + tid / L2;
        const bool act = li < ng * Kz;
        const int j = act ? li / Kz : 0, z = act ? li - (li / Kz) * Kz : 0;
        C* row = planes + (j * N3 + z) * PP;
        C v[M2];
        if (act) split_load_head<N2>(v, row, 1, Ky);
        __syncwarp();
        if (act) {
          split_fwd<N2>(v, l);
#pragma unroll
          for (int m = 0; m < M2; ++m) row[L2 * m + l] = v[m];
        }
      }
    }
    __syncthreads();
    // z: forward, Hadamard with the slab, inverse; columns (j, y < n2)
    {
      const int l = tid % L3;
#pragma unroll 1
      for (int base = 0; base < ng * N2; base += NT / L3) {
        const int li = base + tid / L3;
        const bool act = li < ng * N2;
        const int j = act ? li / N2 : 0, col = act ? li % N2 : 0;
        C* cl = planes + j * N3 * PP + col;
        C v[M3];
        if (act) split_load_head<N3>(v, cl, PP, Kz);
        __syncwarp();
        if (act) {
          split_fwd<N3>(v, l);
#pragma unroll
          for (int m = 0; m < M3; ++m) v[m] = cmul(v[m], Tt[(L3 * m + l) * PT + col]);
          split_inv<N3>(v, l);
        }
        split_inv_store<N3>(v, cl, PP, Kz, l, act);
      }
    }
    __syncthreads();
    // inverse y: rows (j, z < Kz), outputs y < Ky
    {
      const int l = tid % L2;
#pragma unroll 1
      for (int base = 0; base < ng * Kz; base += NT / L2) {
        const int li = base + tid / L2;
        const bool act = li < ng * Kz;
        const int j = act ? li / Kz : 0, z = act ? li - (li / Kz) * Kz : 0;
        C* row = planes + (j * N3 + z) * PP;
        C v[M2];
        if (act) {
#pragma unroll
          for (int m = 0; m < M2; ++m) v[m] = row[L2 * m + l];
        }
        __syncwarp();
        if (act) split_inv<N2>(v, l);
        split_inv_store<N2>(v, row, 1, Ky, l, act);
      }
    }
    __syncthreads();
    for (int i = tid; i < ng * fsz; i += NT) {
      const int j = i / fsz, r = i - j * fsz;
      const int z = r / Ky, y = r - z * Ky;
      const size_t f = (size_t)p * P.nf + g0 + j;
      inter[(f * P.n1 + x) * fsz + r] = planes[(j * N3 + z) * PP + y];
    }
  }
}

}  // namespace fmm
