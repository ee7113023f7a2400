// Register / shared-memory FFT building blocks for the translation kernels.
//
// The translation of Eq. 5 takes, per field, a forward 3D DFT of a box grid
// zero-padded to n1 x n2 x n3, a Hadamard product with the FFT'ed operator and
// an inverse 3D DFT of which only the first K_i entries per axis are kept.
// Every axis length n is a power of two with n >= 2K - 1, so on input only the
// first half of a forward line can be non-zero, and of an inverse line only
// the first half of the output is ever used; the routines below prune both.
//
// A line of length N = R1 * R2 is transformed by a team of T = R1 consecutive
// lanes of one warp in two Cooley-Tukey stages over the R2-strided index:
//   n = a + R2 b  (a < R2, b < R1),    k = c + R1 d  (c < R1, d < R2)
//   X[c + R1 d] = sum_a W_N^{a c} W_R2^{a d} [ sum_b x[a + R2 b] W_R1^{b c} ]
// Stage 1: lane t owns a in {t, t + T, ...}: an R1-point DFT over b, times the
// twiddle W_N^{a c}, written to the team's exchange buffer.  Stage 2: lane t
// owns c = t: an R2-point DFT over a.  Forward transforms use
// W = exp(-2 pi i / N), inverse ones exp(+2 pi i / N), unnormalised.
//
// The stage-2 output of a forward line (lane t holds X[t + R1 d], d < R2) is
// exactly the stage-1 input of an inverse line of the swapped shape
// (R1' = R2, R2' = R1, lane t owns a' = t), which lets the z-lines run
// forward -> Hadamard -> inverse without leaving registers (`line_conv`).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace fmm {

// ---------------------------------------------------------------------------
// complex helpers (float2 / double2)
// ---------------------------------------------------------------------------
template <typename R> struct cx_of;
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<double> { using type = double2; };
template <typename R> using cx = typename cx_of<R>::type;

template <typename C> struct real_of;
template <> struct real_of<float2> { using type = float; };
template <> struct real_of<double2> { using type = double; };

template <typename C>
__device__ __forceinline__ C mk(typename real_of<C>::type a, typename real_of<C>::type b) {
  C r; r.x = a; r.y = b; return r;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk<C>(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk<C>(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk<C>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk<C>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// acc += a * b
template <typename C> __device__ __forceinline__ void cfma(C& acc, C a, C b) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
}
template <typename C> __device__ __forceinline__ C czero() { return mk<C>(0, 0); }

// complex64 sums and differences as one packed two-lane FP32 instruction
// (add/sub .f32x2) instead of two scalar ones
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "add.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
  float2 r;
  asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
      "mov.b64 ra, {%2, %3};\n\tmov.b64 rb, {%4, %5};\n\t"
      "sub.rn.f32x2 rd, ra, rb;\n\tmov.b64 {%0, %1}, rd;\n\t}"
      : "=f"(r.x), "=f"(r.y)
      : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
  return r;
}

// v times the table twiddle w = exp(-2 pi i m / N): S = -1 uses w, S = +1 conj(w)
template <int S, typename C> __device__ __forceinline__ C twmul(C v, C w) {
  if constexpr (S < 0) return cmul(v, w); else return cmulc(v, w);
}

// ---------------------------------------------------------------------------
// compile-time twiddles: cos / sin of 2 pi m / N by Taylor series evaluated
// by the compiler, with the angle folded into [0, pi/4] by exact symmetries
// ---------------------------------------------------------------------------
constexpr double kPi = 3.14159265358979323846264338327950288;

constexpr double taylor_sin(double x) {
  double term = x, sum = x;
  for (int k = 1; k < 14; ++k) { term *= -x * x / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
  return sum;
}
constexpr double taylor_cos(double x) {
  double term = 1.0, sum = 1.0;
  for (int k = 1; k < 14; ++k) { term *= -x * x / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
  return sum;
}
// angle 2 pi m / N in [0, pi/2] (4m <= N)
constexpr double ct_cos_q(int m, int N) {
  return (8 * m > N) ? taylor_sin(2.0 * kPi * (N - 4 * m) / (4.0 * N)) : taylor_cos(2.0 * kPi * m / N);
}
constexpr double ct_sin_q(int m, int N) {
  return (8 * m > N) ? taylor_cos(2.0 * kPi * (N - 4 * m) / (4.0 * N)) : taylor_sin(2.0 * kPi * m / N);
}
constexpr int ct_mod(int m, int N) { return ((m % N) + N) % N; }
// cos(2 pi m / N): cos(2pi - t) = cos t, cos(pi - t) = -cos t
constexpr double ct_cos(int m, int N) {
  return (2 * ct_mod(m, N) > N) ? ct_cos(N - ct_mod(m, N), N)
         : (4 * ct_mod(m, N) > N) ? -ct_cos_q(N - 2 * ct_mod(m, N), 2 * N)
                                  : ct_cos_q(ct_mod(m, N), N);
}
// sin(2 pi m / N): sin(2pi - t) = -sin t, sin(pi - t) = sin t
constexpr double ct_sin(int m, int N) {
  return (2 * ct_mod(m, N) > N) ? -ct_sin(N - ct_mod(m, N), N)
         : (4 * ct_mod(m, N) > N) ? ct_sin_q(N - 2 * ct_mod(m, N), 2 * N)
                                  : ct_sin_q(ct_mod(m, N), N);
}

// v * exp(S * 2 pi i M / N)
template <int N, int M, int S, typename C>
__device__ __forceinline__ C twiddle_ct(C v) {
  using R = typename real_of<C>::type;
  constexpr int m = ct_mod(M, N);
  if constexpr (m == 0) {
    return v;
  } else if constexpr (4 * m == N) {            // factor = i S
    return (S > 0) ? mk<C>(-v.y, v.x) : mk<C>(v.y, -v.x);
  } else if constexpr (2 * m == N) {            // factor = -1
    return mk<C>(-v.x, -v.y);
  } else if constexpr (4 * m == 3 * N) {        // factor = -i S
    return (S > 0) ? mk<C>(v.y, -v.x) : mk<C>(-v.y, v.x);
  } else if constexpr (8 * m == N || 8 * m == 3 * N || 8 * m == 5 * N || 8 * m == 7 * N) {
    // factor = (c + i s) sqrt(1/2) with c, s = +-1
    constexpr R h = (R)0.70710678118654752440084436210485;
    constexpr R c = (R)(ct_cos(m, N) > 0 ? 1 : -1);
    constexpr R s = (R)(S * (ct_sin(m, N) > 0 ? 1 : -1));
    return mk<C>(h * (c * v.x - s * v.y), h * (c * v.y + s * v.x));
  } else {
    constexpr R c = (R)ct_cos(m, N);
    constexpr R s = (R)(S * ct_sin(m, N));
    return mk<C>(v.x * c - v.y * s, v.x * s + v.y * c);
  }
}

// ---------------------------------------------------------------------------
// In-register DFT of length N (power of two) by radix-2 decimation in time,
// fully unrolled: X[k] = sum_n x[n] exp(S 2 pi i n k / N).  Only the first NZ
// inputs are read; the others are taken as zero.
// ---------------------------------------------------------------------------
template <int N, int NZ, int S, int K = 0, typename C>
__device__ __forceinline__ void dft_combine(C* x, const C* e, const C* o);

template <int N, int NZ, int S, typename C>
__device__ __forceinline__ void dft(C* x) {
  if constexpr (NZ <= 0) {
#pragma unroll
    for (int k = 0; k < N; ++k) x[k] = czero<C>();
  } else if constexpr (N == 1) {
    return;
  } else if constexpr (NZ == 1) {
#pragma unroll
    for (int k = 1; k < N; ++k) x[k] = x[0];
  } else {
    constexpr int H = N / 2;
    C e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) {
      if (2 * i < NZ) e[i] = x[2 * i];
      if (2 * i + 1 < NZ) o[i] = x[2 * i + 1];
    }
    dft<H, (NZ + 1) / 2, S>(e);
    dft<H, NZ / 2, S>(o);
    dft_combine<N, NZ, S, 0>(x, e, o);
  }
}

template <int N, int NZ, int S, int K, typename C>
__device__ __forceinline__ void dft_combine(C* x, const C* e, const C* o) {
  if constexpr (K < N / 2) {
    C t = twiddle_ct<N, K, S>(o[K]);
    x[K] = cadd(e[K], t);
    x[K + N / 2] = csub(e[K], t);
    dft_combine<N, NZ, S, K + 1>(x, e, o);
  }
}

// w[c] = w1^c for c < CNT (w[0] = 1), by repeated squaring / multiplication
// (depth log2 CNT): the stage-1 twiddles W^(a c) of one lane from the single
// table value W^a, trading CNT - 2 shared-memory loads for complex products.
template <int CNT, typename C>
__device__ __forceinline__ void twiddle_powers(C w1, C* w) {
  w[0] = mk<C>(1, 0);
  if constexpr (CNT > 1) w[1] = w1;
#pragma unroll
  for (int c = 2; c < CNT; ++c) w[c] = (c % 2 == 0) ? cmul(w[c / 2], w[c / 2]) : cmul(w[c - 1], w1);
}

// ---------------------------------------------------------------------------
// Line shapes: N = R1 * R2 with R1 <= R2, a team of T = R1 lanes per line.
// ---------------------------------------------------------------------------
template <int N> struct LineCfg;
template <> struct LineCfg<4> { static constexpr int R1 = 2, R2 = 2; };
template <> struct LineCfg<8> { static constexpr int R1 = 2, R2 = 4; };
template <> struct LineCfg<16> { static constexpr int R1 = 4, R2 = 4; };
template <> struct LineCfg<32> { static constexpr int R1 = 4, R2 = 8; };
template <> struct LineCfg<64> { static constexpr int R1 = 8, R2 = 8; };
template <> struct LineCfg<128> { static constexpr int R1 = 8, R2 = 16; };
template <> struct LineCfg<256> { static constexpr int R1 = 16, R2 = 16; };

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int N> struct Line {
  static constexpr int R1 = LineCfg<N>::R1, R2 = LineCfg<N>::R2;
  static constexpr int T = R1;                  // lanes per line
  static constexpr int TPW = 32 / T;            // lines per warp
  static constexpr int XT = N + R2;             // exchange elements per team
  static constexpr int XW = TPW * XT;           // exchange elements per warp
  static constexpr int LPI = kWarps * TPW;      // lines per block iteration
  // spacing of the lines a warp's teams work on; spreads shared-memory banks
  static constexpr int SP = (T < kWarps) ? T : kWarps;
  static_assert(R1 * R2 == N && R1 <= R2 && R2 % R1 == 0, "bad line shape");
};

// Which line of a block iteration this lane's team works on, its lane in the
// team, and its exchange buffer.
template <int N> struct TeamPos {
  int line, t;
  __device__ __forceinline__ TeamPos() {
    using L = Line<N>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = lane / L::T;
    t = lane % L::T;
    line = (w % L::SP) + L::SP * k + L::SP * L::TPW * (w / L::SP);
  }
  template <typename C> __device__ __forceinline__ C* xs(C* xs_block) const {
    using L = Line<N>;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    return xs_block + w * L::XW + (lane / L::T) * L::XT;
  }
};

// One line transform.  Elements at ln[i * es].  IN_HALF: only i < N/2 are
// read (the rest are zero).  Outputs with index < keep are written back.
// Every lane of the warp must call this (active = false lanes only sync).
template <int N, int S, bool IN_HALF, typename C>
__device__ __forceinline__ void line_fft(C* ln, int es, C* xs, const C* tw, int t, bool active,
                                         int keep, const C* wpre = nullptr) {
  using L = Line<N>;
  constexpr int R1 = L::R1, R2 = L::R2, T = L::T;
  constexpr int A = R2 / T;
  constexpr int NZ1 = IN_HALF ? R1 / 2 : R1;
  constexpr bool kSquare = R1 == R2 && A == 1;   // wpre: as in line_conv
  if (active) {
#pragma unroll
    for (int i = 0; i < A; ++i) {
      const int a = t + T * i;
      C v[R1];
#pragma unroll
      for (int b = 0; b < NZ1; ++b) v[b] = ln[(a + R2 * b) * es];
      dft<R1, NZ1, S>(v);
      C w[R1];
      if (kSquare && wpre) {
#pragma unroll
        for (int c = 0; c < R1; ++c) w[c] = wpre[c];
      } else {
        twiddle_powers<R1>(tw[a], w);
      }
      xs[a] = v[0];
#pragma unroll
      for (int c = 1; c < R1; ++c) xs[c * (R2 + 1) + a] = twmul<S>(v[c], w[c]);
    }
  }
  __syncwarp();
  if (active) {
    const int c = t;
    C v[R2];
#pragma unroll
    for (int a = 0; a < R2; ++a) v[a] = xs[c * (R2 + 1) + a];
    dft<R2, R2, S>(v);
#pragma unroll
    for (int d = 0; d < R2; ++d) {
      const int k = c + R1 * d;
      if (k < keep) ln[k * es] = v[d];
    }
  }
  __syncwarp();
}

// Forward transform of a half-filled line, Hadamard product with op[k * op_es]
// (k < N), inverse transform; outputs with index < keep (<= N) written back.
// OP_EARLY: the lane's operator values are loaded before the forward
// transform, so that their latency overlaps it (op in global memory; it costs
// 2 R2 registers across the transform); otherwise when they are used.
// wpre: for square shapes (R1 = R2, one stage-1 DFT per lane) the lane's
// twiddles W^(t c), c < R1, computed once by the caller (line_twiddles) and
// shared by the forward and the inverse stage 1; null: computed here.
template <int N, bool OP_EARLY = false, typename C>
__device__ __forceinline__ void line_conv(C* ln, int es, C* xs, const C* tw, const C* op, int op_es,
                                          int t, bool active, int keep, const C* wpre = nullptr) {
  using L = Line<N>;
  constexpr int R1 = L::R1, R2 = L::R2, T = L::T;
  constexpr int A = R2 / T;          // forward stage-1 DFTs per lane
  constexpr int B2 = R2 / T;         // inverse stage-2 DFTs per lane
  constexpr int NZ1 = R1 / 2;
  constexpr bool kSquare = R1 == R2 && A == 1;
  C opv[OP_EARLY ? R2 : 1];
  if constexpr (OP_EARLY) {
    if (active) {
#pragma unroll
      for (int d = 0; d < R2; ++d) opv[d] = op[(t + R1 * d) * op_es];
    }
  }
  // forward stage 1
  if (active) {
#pragma unroll
    for (int i = 0; i < A; ++i) {
      const int a = t + T * i;
      C v[R1];
#pragma unroll
      for (int b = 0; b < NZ1; ++b) v[b] = ln[(a + R2 * b) * es];
      dft<R1, NZ1, -1>(v);
      C w[R1];
      if (kSquare && wpre) {
#pragma unroll
        for (int c = 0; c < R1; ++c) w[c] = wpre[c];
      } else {
        twiddle_powers<R1>(tw[a], w);
      }
      xs[a] = v[0];
#pragma unroll
      for (int c = 1; c < R1; ++c) xs[c * (R2 + 1) + a] = twmul<-1>(v[c], w[c]);
    }
  }
  __syncwarp();
  C v[R2];
  if (active) {
#pragma unroll
    for (int a = 0; a < R2; ++a) v[a] = xs[t * (R2 + 1) + a];
  }
  __syncwarp();
  if (active) {
    // forward stage 2: v[d] = X[t + R1 d]
    dft<R2, R2, -1>(v);
#pragma unroll
    for (int d = 0; d < R2; ++d) {
      if constexpr (OP_EARLY) v[d] = cmul(v[d], opv[d]);
      else v[d] = cmul(v[d], op[(t + R1 * d) * op_es]);
    }
    // inverse stage 1 of the swapped shape (R1' = R2, R2' = R1): a' = t,
    // inputs x[t + R1 b'] = v[b'] for b' < R2
    dft<R2, R2, +1>(v);
    {
      C w[R2];
      if (kSquare && wpre) {
#pragma unroll
        for (int c = 0; c < R2; ++c) w[c] = wpre[c];
      } else {
        twiddle_powers<R2>(tw[t], w);
      }
      xs[t] = v[0];
#pragma unroll
      for (int c = 1; c < R2; ++c) xs[c * (R1 + 1) + t] = twmul<+1>(v[c], w[c]);
    }
  }
  __syncwarp();
  if (active) {
    // inverse stage 2: c' = t + T j, R1-point DFTs over a' < R1;
    // outputs k = c' + R2 d'
#pragma unroll
    for (int j = 0; j < B2; ++j) {
      const int c = t + T * j;
      C u[R1];
#pragma unroll
      for (int a = 0; a < R1; ++a) u[a] = xs[c * (R1 + 1) + a];
      dft<R1, R1, +1>(u);
#pragma unroll
      for (int d = 0; d < R1; ++d) {
        const int k = c + R2 * d;
        if (k < keep) ln[k * es] = u[d];
      }
    }
  }
  __syncwarp();
}

// ---------------------------------------------------------------------------
// Small complex GEMM on shared-memory operands, all threads of the block:
//   Cm[m * ldc + n] = scale * sum_k A[m * lda + k] * B[k * ldb + n]
// Each warp computes TM rows x (32 TN) columns at a time; lane l owns columns
// n0 + l + 32 j, so B reads are conflict-free and A reads are broadcasts.
// Cm may point to shared or global memory.
// ---------------------------------------------------------------------------
template <int TM, int TN, typename C>
__device__ __forceinline__ void block_cgemm(int M, int N, int K, const C* A, int lda, const C* B,
                                            int ldb, C* Cm, int ldc,
                                            typename real_of<C>::type scale) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nrb = (M + TM - 1) / TM, ncb = (N + 32 * TN - 1) / (32 * TN);
  for (int item = w; item < nrb * ncb; item += kWarps) {
    const int m0 = (item / ncb) * TM, n0 = (item % ncb) * (32 * TN);
    C acc[TM][TN];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TN; ++j) acc[i][j] = czero<C>();
    for (int k = 0; k < K; ++k) {
      C b[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + lane + 32 * j;
        b[j] = (n < N) ? B[k * ldb + n] : czero<C>();
      }
#pragma unroll
      for (int i = 0; i < TM; ++i) {
        const int m = m0 + i;
        const C a = (m < M) ? A[m * lda + k] : czero<C>();
#pragma unroll
        for (int j = 0; j < TN; ++j) cfma(acc[i][j], a, b[j]);
      }
    }
#pragma unroll
    for (int i = 0; i < TM; ++i) {
      const int m = m0 + i;
      if (m >= M) continue;
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        const int n = n0 + lane + 32 * j;
        if (n < N) Cm[m * ldc + n] = mk<C>(acc[i][j].x * scale, acc[i][j].y * scale);
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Complex GEMM with general strides, all threads of the block, operands and
// result anywhere (shared or global memory):
//   Cm[m * ldc + n] = scale * sum_k A[m * sam + k * sak] * B[k * sbk + n * sbn]
// Each thread computes outputs (m, n) with n = lane + 32 j of a 4-row group.
// ---------------------------------------------------------------------------
template <typename C>
__device__ __forceinline__ void block_cgemm_strided(int M, int N, int K, const C* A, long sam, long sak,
                                                    const C* B, long sbk, long sbn, C* Cm, long ldc,
                                                    typename real_of<C>::type scale) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int nrb = (M + 3) / 4, ncb = (N + 31) / 32;
  for (int item = w; item < nrb * ncb; item += nw) {
    const int m0 = (item / ncb) * 4, n = (item % ncb) * 32 + lane;
    C acc[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i] = czero<C>();
    if (n < N) {
      for (int k = 0; k < K; ++k) {
        const C b = B[k * sbk + n * sbn];
#pragma unroll
        for (int i = 0; i < 4; ++i)
          if (m0 + i < M) cfma(acc[i], A[(m0 + i) * sam + k * sak], b);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
        if (m0 + i < M) Cm[(m0 + i) * ldc + n] = mk<C>(acc[i].x * scale, acc[i].y * scale);
    }
  }
}

}  // namespace fmm
