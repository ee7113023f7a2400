// Complex 64 x 64 GEMM tile on the 5th-generation tensor cores (tcgen05) in
// 3xTF32 split precision with FP32 accumulation in tensor memory (TMEM), for
// the operator restores (Sec. II.C): all threads of a 256-thread block call
// tc_cgemm64.
//
// Complex product C = A B (A: M x K, B: K x N, M, N <= 64) as one real MMA of
// shape 128 x 128 x K per K step:
//   A' = [Re A ; Im A]   (rows 0..63 real parts, 64..127 imaginary parts)
//   B' = [Re B , Im B]   (columns 0..63 real parts, 64..127 imaginary parts)
//   D  = A' B' = [[ReA ReB, ReA ImB], [ImA ReB, ImA ImB]]
//   Re C = D[m][n] - D[64+m][64+n],   Im C = D[m][64+n] + D[64+m][n]
// Each FP32 operand x is split into tf32 parts x = big + small (big = x rounded
// to tf32, small = the rounded remainder) and D accumulates big*big +
// small*big + big*small: the dropped small*small term and the rounding of
// `small` leave a relative error near 2^-21, the FP32 level.
//
// BF16 variant (template flag): the parts are bf16 (x = hi + lo, lo = the
// bf16 rounding of x - hi), products of kind::f16 with BF16 inputs; a 32-bit
// staging word holds two consecutive K elements, so the same staging layout
// covers twice the K per chunk.  Relative error near 2^-16 per product.
//
// Operands are staged through shared memory in chunks of kTcKC along K, in
// the no-swizzle K-major canonical layout of tcgen05: 8-row x 16-byte core
// matrices, the 4 core matrices of a chunk's K extent adjacent (LBO = 128 B),
// 8-row groups 512 B apart (SBO).  B' is stored transposed (N' x K, K-major).
// One elected thread issues the MMAs and commits them to an mbarrier; warp 0
// waits on it (bounded) while the other warps sleep in a block barrier, so the
// wait takes no shared-memory bandwidth from a co-resident block.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fmm {

constexpr int kTcKC = 16;                              // complex K per chunk
constexpr int kTcTileFloats = 128 * kTcKC;             // one 128 x KC operand split
constexpr size_t kTcSmemBytes = 4 * kTcTileFloats * sizeof(float);  // A big/small, B big/small
constexpr int kTcCols = 128;                           // TMEM columns of D
constexpr unsigned kTcWaitLimit = 1u << 24;            // mbarrier poll limit

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm volatile("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// float offset of element (row, k) of a 128 x kTcKC tile in the canonical
// K-major layout (core matrix = 8 rows x 4 floats)
__device__ __forceinline__ int tc_off(int row, int k) {
  return (((row >> 3) * (kTcKC / 4) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

// bytes of operand staging for chunks of KC complex K (A big/small, B big/small)
template <int KC>
constexpr size_t tc_smem_bytes() {
  return 4 * 128 * (size_t)KC * sizeof(float);
}

// shared-memory matrix descriptor: no swizzle, LBO 128 B (K direction), SBO
// between 8-row groups (KC / 4 core matrices of 128 B each), version 1
template <int KC = kTcKC>
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
  const uint64_t lbo = 128, sbo = (KC / 4) * 128;
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32, D in F32, A and B K-major, M = N = 128
__host__ __device__ constexpr uint32_t tc_idesc_tf32_128x128() {
  return (1u << 4)                 // D format F32
         | (2u << 7)               // A format TF32
         | (2u << 10)              // B format TF32
         | ((128u >> 3) << 17)     // N >> 3
         | ((128u >> 4) << 24);    // M >> 4
}

// instruction descriptor of kind::f16 with BF16 inputs, D in F32, A and B
// K-major, M = N = 128
__host__ __device__ constexpr uint32_t tc_idesc_bf16_128x128() {
  return (1u << 4)                 // D format F32
         | (1u << 7)               // A format BF16
         | (1u << 10)              // B format BF16
         | ((128u >> 3) << 17)     // N >> 3
         | ((128u >> 4) << 24);    // M >> 4
}

__device__ __forceinline__ void tc_mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// hi and lo bf16 parts of two values, each pair packed into one word (first
// value in the low half, the lower address)
__device__ __forceinline__ void bf16_split2(float a, float b, uint32_t& hi, uint32_t& lo) {
  const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
  const float2 hf = __bfloat1622float2(h);
  const __nv_bfloat162 l = __floats2bfloat162_rn(a - hf.x, b - hf.y);
  hi = *reinterpret_cast<const uint32_t*>(&h);
  lo = *reinterpret_cast<const uint32_t*>(&l);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
      :
      : "r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}

// Wait for phase `parity` of the mbarrier to complete; false after the poll
// limit.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  for (unsigned it = 0; it < kTcWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// TMEM allocation by one full warp; the address lands in *slot (shared).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// 16 consecutive FP32 columns of this thread's TMEM lane (32x32b shape).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// Per-block state of the tensor-core GEMMs: TMEM address, mbarrier and its
// phase, staged in shared memory by tc_setup.
struct TcState {
  float* buf;          // 4 x kTcTileFloats floats: A big, A small, B big, B small
  uint32_t mbar;       // shared address of the mbarrier
  uint32_t tmem;       // TMEM base address of D
  uint32_t phase;      // parity of the next mbarrier phase
  bool ok;             // false once a wait ran out (results invalid)
  bool single;         // 3xTF32 path: one TF32 product (big x big) only
  uint32_t mbar2;      // second mbarrier (pipelined GEMM: odd chunks), 0 if none
  uint32_t phase2;     // parity of its next phase
};

// Block-wide set-up: `buf` (kTcSmemBytes, 16-byte aligned) holds the operand
// chunks, `bar` is the mbarrier (8 bytes of shared memory that nothing else
// uses while the state lives; `bar2` a second one for tc_cgemm64_pipe) and
// `slot` receives the TMEM address.  Warp 0
// allocates kTcCols columns.  All threads call it.
__device__ __forceinline__ TcState tc_setup(void* buf, uint64_t* bar, uint32_t* slot, uint64_t* bar2 = nullptr) {
  TcState s;
  s.buf = reinterpret_cast<float*>(buf);
  s.mbar = smem_u32(bar);
  s.mbar2 = bar2 ? smem_u32(bar2) : 0u;
  s.phase2 = 0;
  if (threadIdx.x == 0) {
    mbar_init(s.mbar, 1);
    if (bar2) mbar_init(s.mbar2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if ((threadIdx.x >> 5) == 0) tmem_alloc(slot, kTcCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  s.tmem = *slot;
  s.phase = 0;
  s.ok = true;
  s.single = false;
  return s;
}

// Block-wide tear-down: warp 0 frees the TMEM columns.  All threads call it,
// after their last TMEM access.
__device__ __forceinline__ void tc_teardown(const TcState& s) {
  tc_fence_before();
  __syncthreads();
  if ((threadIdx.x >> 5) == 0) {
    tc_fence_after();
    tmem_dealloc(s.tmem, kTcCols);
  }
}

// Epilogue shared by the GEMM variants: D (128 x 128 FP32 in TMEM) to the
// complex C tile.
template <bool C_GLOBAL>
__device__ __forceinline__ void tc_epilogue(TcState& s, int M, int N, float2* C, int ldc, float scale) {
  const int tid = threadIdx.x;
  // epilogue: lanes m (warps 0, 1 and 4, 5) hold the ReA rows, lanes 64 + m
  // (warps 2, 3 and 6, 7) the ImA rows; warps w and w + 4 split the columns.
  const int w = tid >> 5, q = w & 3, half = w >> 2;
  const int row = q * 32 + (tid & 31);
  const uint32_t lane_addr = s.tmem + ((uint32_t)(q * 32) << 16);
  float v[16];
  if constexpr (C_GLOBAL) {
    // combine in the (now idle) operand buffer, a 64 x 64 complex tile with
    // columns XOR-swizzled by the row, then copy to C with consecutive
    // threads on consecutive columns
    float2* T = reinterpret_cast<float2*>(s.buf);
    if (q < 2) {
      const int m = row;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld16(lane_addr + half * 64 + c * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float2* t = &T[m * 64 + ((c * 16 + j) ^ (m & 31))];
          if (half == 0) t->x = v[j];      // ReA ReB
          else t->y = v[j];                // ReA ImB
        }
      }
    }
    __syncthreads();
    if (q >= 2) {
      const int m = row - 64;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld16(lane_addr + half * 64 + c * 16, v);
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          float2* t = &T[m * 64 + ((c * 16 + j) ^ (m & 31))];
          if (half == 0) t->y += v[j];     // + ImA ReB
          else t->x -= v[j];               // - ImA ImB
        }
      }
    }
    tc_fence_before();
    __syncthreads();
    for (int i = tid; i < M * 64; i += 256) {
      const int m = i >> 6, n = i & 63;
      if (n < N) {
        const float2 t = T[m * 64 + (n ^ (m & 31))];
        C[m * ldc + n] = make_float2(t.x * scale, t.y * scale);
      }
    }
    __syncthreads();
  } else {
    if (q < 2) {
      const int m = row;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld16(lane_addr + half * 64 + c * 16, v);
        if (m < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c * 16 + j;
            if (n < N) {
              if (half == 0) C[m * ldc + n].x = v[j];   // ReA ReB
              else C[m * ldc + n].y = v[j];              // ReA ImB
            }
          }
        }
      }
    }
    __syncthreads();
    if (q >= 2) {
      const int m = row - 64;
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        tmem_ld16(lane_addr + half * 64 + c * 16, v);
        if (m < M) {
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int n = c * 16 + j;
            if (n < N) {
              if (half == 0) C[m * ldc + n].y = (C[m * ldc + n].y + v[j]) * scale;   // + ImA ReB
              else C[m * ldc + n].x = (C[m * ldc + n].x - v[j]) * scale;             // - ImA ImB
            }
          }
        }
      }
    }
    tc_fence_before();
    __syncthreads();
  }
}

// BF16x3 variant of tc_cgemm64 (see the header comment): word i of a staging
// tile holds K elements 2 kw and 2 kw + 1 of row m, with (m, kw) placed as the
// TF32 variant places (m, k); a chunk covers kTcKC words = 2 kTcKC elements.
template <bool C_GLOBAL, typename FA, typename FB>
__device__ __forceinline__ void tc_cgemm64_bf16(TcState& s, int M, int N, int K, FA a_of, FB b_of, float2* C,
                                                int ldc, float scale) {
  const int tid = threadIdx.x;
  uint32_t* Ab = reinterpret_cast<uint32_t*>(s.buf);
  uint32_t* As = Ab + kTcTileFloats;
  uint32_t* Bb = As + kTcTileFloats;
  uint32_t* Bs = Bb + kTcTileFloats;
  constexpr uint32_t idesc = tc_idesc_bf16_128x128();
  constexpr int KE = 2 * kTcKC;                    // K elements per chunk
  const int nchunks = (K + KE - 1) / KE;
  constexpr int kPer = 64 * kTcKC / 256;
  float2 va[2 * kPer], vb[2 * kPer];
  auto gather = [&](int k0) {
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + 256 * j;
      const int cm = i >> 5, w = i & 31;
      const int m = (cm / (kTcKC / 4)) * 8 + (w >> 2);
      const int gk = k0 + 2 * ((cm % (kTcKC / 4)) * 4 + (w & 3));
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        va[2 * j + e] = (gk + e < K && m < M) ? a_of(m, gk + e) : make_float2(0.f, 0.f);
        vb[2 * j + e] = (gk + e < K && m < N) ? b_of(gk + e, m) : make_float2(0.f, 0.f);
      }
    }
  };
  gather(0);
  for (int ch = 0; ch < nchunks; ++ch) {
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int o0 = tid + 256 * j, o1 = o0 + 64 * kTcKC;
      const float2 a0 = va[2 * j], a1 = va[2 * j + 1], b0 = vb[2 * j], b1 = vb[2 * j + 1];
      uint32_t hi, lo;
      bf16_split2(a0.x, a1.x, hi, lo);
      Ab[o0] = hi;
      As[o0] = lo;
      bf16_split2(a0.y, a1.y, hi, lo);
      Ab[o1] = hi;
      As[o1] = lo;
      bf16_split2(b0.x, b1.x, hi, lo);
      Bb[o0] = hi;
      Bs[o0] = lo;
      bf16_split2(b0.y, b1.y, hi, lo);
      Bb[o1] = hi;
      Bs[o1] = lo;
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ab = smem_u32(Ab), as = smem_u32(As), bb = smem_u32(Bb), bs = smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < kTcKC / 8; ++ks) {
        const uint32_t step = ks * 2 * 128;        // two core matrices (16 bf16) along K
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        tc_mma_bf16(s.tmem, tc_desc(ab + step), tc_desc(bb + step), idesc, acc0);
        tc_mma_bf16(s.tmem, tc_desc(as + step), tc_desc(bb + step), idesc, 1u);
        tc_mma_bf16(s.tmem, tc_desc(ab + step), tc_desc(bs + step), idesc, 1u);
      }
      tc_commit(s.mbar);
    }
    if (ch + 1 < nchunks) gather((ch + 1) * KE);
    bool timeout = false;
    if (tid < 32) timeout = !mbar_wait(s.mbar, s.phase);
    if (__syncthreads_or(timeout)) s.ok = false;
    s.phase ^= 1u;
    tc_fence_after();
  }
  tc_epilogue<C_GLOBAL>(s, M, N, C, ldc, scale);
}

// C[m * ldc + n] = scale * sum_k A(m, k) B(k, n) for m < M, n < N (M, N <= 64)
// with A(m, k), B(k, n) complex (float2) supplied by the functors.  Every
// thread of the 256-thread block calls it.  C_GLOBAL: C is in global memory,
// so the epilogue combines the quadrants in shared memory and writes C once,
// coalesced; otherwise C (shared memory) is written directly, one row per lane.
// KC: complex K per staged chunk (3xTF32 path); `s.buf` must hold
// tc_smem_bytes<KC>().  Larger chunks halve the round trips of long
// contractions at the price of registers and shared memory.
template <bool C_GLOBAL, bool BF16 = false, int KC = kTcKC, typename FA, typename FB>
__device__ __forceinline__ void tc_cgemm64(TcState& s, int M, int N, int K, FA a_of, FB b_of, float2* C,
                                           int ldc, float scale) {
  if constexpr (BF16) {
    tc_cgemm64_bf16<C_GLOBAL>(s, M, N, K, a_of, b_of, C, ldc, scale);
    return;
  }
  const int tid = threadIdx.x;
  uint32_t* Ab = reinterpret_cast<uint32_t*>(s.buf);
  constexpr int kTile = 128 * KC;
  uint32_t* As = Ab + kTile;
  uint32_t* Bb = As + kTile;
  uint32_t* Bs = Bb + kTile;
  constexpr uint32_t idesc = tc_idesc_tf32_128x128();
  const int nchunks = (K + KC - 1) / KC;
  // Element i of the first 64 rows of a chunk sits at float i of the tile:
  // core matrix i / 32 (row group, K group), row (i % 32) / 4, column i % 4;
  // the second 64 rows follow 1024 floats later.  Each thread owns i = tid +
  // 256 j (j < 4); consecutive threads write consecutive words.
  constexpr int kPer = 64 * KC / 256;
  float2 va[kPer], vb[kPer];
  auto gather = [&](int k0) {
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + 256 * j;
      const int cm = i >> 5, w = i & 31;
      const int m = (cm / (KC / 4)) * 8 + (w >> 2);
      const int gk = k0 + (cm % (KC / 4)) * 4 + (w & 3);
      va[j] = (gk < K && m < M) ? a_of(m, gk) : make_float2(0.f, 0.f);
      vb[j] = (gk < K && m < N) ? b_of(gk, m) : make_float2(0.f, 0.f);
    }
  };
  gather(0);
  for (int ch = 0; ch < nchunks; ++ch) {
    // stage chunk: A' rows m (real) and 64 + m (imaginary); B'^T rows n
    // (real) and 64 + n (imaginary), K contiguous
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int o0 = tid + 256 * j, o1 = o0 + 64 * KC;
      const float2 a = va[j], b = vb[j];
      const uint32_t arb = to_tf32(a.x), aib = to_tf32(a.y);
      const uint32_t brb = to_tf32(b.x), bib = to_tf32(b.y);
      Ab[o0] = arb;
      Ab[o1] = aib;
      Bb[o0] = brb;
      Bb[o1] = bib;
      if (!s.single) {
        As[o0] = to_tf32(a.x - __uint_as_float(arb));
        As[o1] = to_tf32(a.y - __uint_as_float(aib));
        Bs[o0] = to_tf32(b.x - __uint_as_float(brb));
        Bs[o1] = to_tf32(b.y - __uint_as_float(bib));
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ab = smem_u32(Ab), as = smem_u32(As), bb = smem_u32(Bb), bs = smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < KC / 8; ++ks) {
        const uint32_t step = ks * 2 * 128;        // two core matrices along K
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        tc_mma(s.tmem, tc_desc<KC>(ab + step), tc_desc<KC>(bb + step), idesc, acc0);
        if (!s.single) {
          tc_mma(s.tmem, tc_desc<KC>(as + step), tc_desc<KC>(bb + step), idesc, 1u);
          tc_mma(s.tmem, tc_desc<KC>(ab + step), tc_desc<KC>(bs + step), idesc, 1u);
        }
      }
      tc_commit(s.mbar);
    }
    // the next chunk's loads overlap the MMAs of this one
    if (ch + 1 < nchunks) gather((ch + 1) * KC);
    // warp 0 polls the mbarrier (each poll is a shared-memory operation);
    // the other warps sleep in the barrier, which also shares the outcome
    bool timeout = false;
    if (tid < 32) timeout = !mbar_wait(s.mbar, s.phase);
    if (__syncthreads_or(timeout)) s.ok = false;
    s.phase ^= 1u;
    tc_fence_after();
  }
  tc_epilogue<C_GLOBAL>(s, M, N, C, ldc, scale);
}

// one complex element (8 bytes) global -> shared, asynchronously; valid =
// false reads nothing and writes zeros
__device__ __forceinline__ void cp_async8_zfill(void* dst, const void* src, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(smem_u32(dst)), "l"(src),
               "r"(valid ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_groups() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------------------
// Pipelined complex 64 x 64 tile (3xTF32 or BF16x3) for long contractions:
// chunks of kPipeK complex K; the raw FP32 operands of chunk ch + 1 are
// copied (cp.async) into one of two ring stages while chunk ch is split, and
// the split goes to one of two staging buffers, so that chunk ch's split
// overlaps chunk ch - 1's MMAs.  Chunk ch's MMAs commit to mbarrier
// (ch even ? s.mbar : s.mbar2); a staging buffer is reused only after the
// MMAs that read it (two chunks earlier) have completed.  A and B are given
// by base pointers and element strides in global memory: A(m, k) =
// A[m am + k ak] (M x K), B(k, n) = B[k bk + n bn] (K x N); elements outside
// M, N or K are zero-filled by the copies.  Ring rows hold kPipeK complex k,
// XOR-swizzled by the row so that the split's reads (8 rows x 4 k per warp)
// and the copies spread over the banks.  Shared memory: s.buf holds the two
// staging buffers (tc_pipe_staging_bytes) and `ring` kPipeRingBytes; s.mbar2
// must be set up.  All threads call it.
// ---------------------------------------------------------------------------
constexpr int kPipeK = 16;
constexpr size_t kPipeRingBytes = 2 * 2 * 64 * (size_t)kPipeK * sizeof(float2);
template <bool BF16>
constexpr size_t tc_pipe_staging_bytes() {
  return 2 * 4 * 128 * (size_t)(BF16 ? kPipeK / 2 : kPipeK) * sizeof(uint32_t);
}

template <bool C_GLOBAL, bool BF16>
__device__ __forceinline__ void tc_cgemm64_pipe(TcState& s, float2* ring, int M, int N, int K, const float2* A,
                                                long long am, long long ak, const float2* B, long long bk,
                                                long long bn, float2* C, int ldc, float scale) {
  constexpr int KE = kPipeK;                        // complex K per chunk
  constexpr int KCW = BF16 ? KE / 2 : KE;           // staging words per row
  constexpr int kTile = 128 * KCW;                  // words per operand part
  constexpr int kStage = 2 * 64 * KE;               // float2 per ring stage
  constexpr uint32_t idesc = BF16 ? tc_idesc_bf16_128x128() : tc_idesc_tf32_128x128();
  const int tid = threadIdx.x, lane = tid & 31;
  const int nchunks = (K + KE - 1) / KE;
  uint32_t* stg0 = reinterpret_cast<uint32_t*>(s.buf);
  auto swz = [](int m, int k) { return m * KE + (k ^ ((m & 3) << 2)); };
  const bool a_rows = am == 1, b_rows = bn == 1;
  auto issue = [&](int ch) {
    if (ch < nchunks) {
      float2* ra = ring + (ch & 1) * kStage;
      float2* rb = ra + 64 * KE;
      const int k0 = ch * KE;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int e = tid + 256 * j, bw = e >> 5;
        const int mr = (bw & 7) * 8 + (lane & 7), kr = (bw >> 3) * 4 + (lane >> 3);
        const int mc = e >> 4, kc = e & 15;
        {
          const int m = a_rows ? mr : mc, k = a_rows ? kr : kc;
          const bool v = m < M && k0 + k < K;
          cp_async8_zfill(ra + swz(m, k), v ? A + m * am + (long long)(k0 + k) * ak : A, v);
        }
        {
          const int n = b_rows ? mr : mc, k = b_rows ? kr : kc;
          const bool v = n < N && k0 + k < K;
          cp_async8_zfill(rb + swz(n, k), v ? B + (long long)(k0 + k) * bk + n * bn : B, v);
        }
      }
    }
    cp_async_commit();                              // one group per chunk, empty or not
  };
  // wait for the MMAs of chunk c (the last commit on its mbarrier)
  auto wait_chunk = [&](int c) {
    const uint32_t bar = (c & 1) ? s.mbar2 : s.mbar;
    uint32_t& ph = (c & 1) ? s.phase2 : s.phase;
    bool timeout = false;
    if (tid < 32) timeout = !mbar_wait(bar, ph);
    if (__syncthreads_or(timeout)) s.ok = false;
    ph ^= 1u;
    tc_fence_after();
  };
  issue(0);
  for (int ch = 0; ch < nchunks; ++ch) {
    issue(ch + 1);                                  // into the stage chunk ch - 1 was split from
    cp_async_wait_groups<1>();                      // this thread's copies of chunk ch
    if (ch >= 2) {
      wait_chunk(ch - 2);                           // its staging buffer is free again
    } else {
      __syncthreads();                              // every thread's copies of chunk ch landed
    }
    const float2* ra = ring + (ch & 1) * kStage;
    const float2* rb = ra + 64 * KE;
    uint32_t* Ab = stg0 + (ch & 1) * 4 * kTile;
    uint32_t* As = Ab + kTile;
    uint32_t* Bb = As + kTile;
    uint32_t* Bs = Bb + kTile;
#pragma unroll
    for (int j = 0; j < 64 * KCW / 256; ++j) {
      const int i = tid + 256 * j;
      const int cm = i >> 5, w = i & 31;
      const int m = (cm / (KCW / 4)) * 8 + (w >> 2);
      const int kw = (cm % (KCW / 4)) * 4 + (w & 3);
      const int o0 = i, o1 = o0 + 64 * KCW;
      if constexpr (BF16) {
        const float2 a0 = ra[swz(m, 2 * kw)], a1 = ra[swz(m, 2 * kw + 1)];
        const float2 b0 = rb[swz(m, 2 * kw)], b1 = rb[swz(m, 2 * kw + 1)];
        uint32_t hi, lo;
        bf16_split2(a0.x, a1.x, hi, lo);
        Ab[o0] = hi;
        As[o0] = lo;
        bf16_split2(a0.y, a1.y, hi, lo);
        Ab[o1] = hi;
        As[o1] = lo;
        bf16_split2(b0.x, b1.x, hi, lo);
        Bb[o0] = hi;
        Bs[o0] = lo;
        bf16_split2(b0.y, b1.y, hi, lo);
        Bb[o1] = hi;
        Bs[o1] = lo;
      } else {
        const float2 a = ra[swz(m, kw)], b = rb[swz(m, kw)];
        const uint32_t arb = to_tf32(a.x), aib = to_tf32(a.y);
        const uint32_t brb = to_tf32(b.x), bib = to_tf32(b.y);
        Ab[o0] = arb;
        Ab[o1] = aib;
        Bb[o0] = brb;
        Bb[o1] = bib;
        if (!s.single) {
          As[o0] = to_tf32(a.x - __uint_as_float(arb));
          As[o1] = to_tf32(a.y - __uint_as_float(aib));
          Bs[o0] = to_tf32(b.x - __uint_as_float(brb));
          Bs[o1] = to_tf32(b.y - __uint_as_float(bib));
        }
      }
    }
    fence_async_smem();
    __syncthreads();
    if (tid == 0) {
      tc_fence_after();
      const uint32_t ab = smem_u32(Ab), as = smem_u32(As), bb = smem_u32(Bb), bs = smem_u32(Bs);
#pragma unroll
      for (int ks = 0; ks < KCW / 8; ++ks) {
        const uint32_t step = ks * 2 * 128;         // two core matrices along K
        const uint32_t acc0 = (ch > 0 || ks > 0) ? 1u : 0u;
        if constexpr (BF16) {
          tc_mma_bf16(s.tmem, tc_desc<KCW>(ab + step), tc_desc<KCW>(bb + step), idesc, acc0);
          tc_mma_bf16(s.tmem, tc_desc<KCW>(as + step), tc_desc<KCW>(bb + step), idesc, 1u);
          tc_mma_bf16(s.tmem, tc_desc<KCW>(ab + step), tc_desc<KCW>(bs + step), idesc, 1u);
        } else {
          tc_mma(s.tmem, tc_desc<KCW>(ab + step), tc_desc<KCW>(bb + step), idesc, acc0);
          if (!s.single) {
            tc_mma(s.tmem, tc_desc<KCW>(as + step), tc_desc<KCW>(bb + step), idesc, 1u);
            tc_mma(s.tmem, tc_desc<KCW>(ab + step), tc_desc<KCW>(bs + step), idesc, 1u);
          }
        }
      }
      tc_commit((ch & 1) ? s.mbar2 : s.mbar);
    }
  }
  cp_async_wait_groups<0>();                        // no copy left in flight
  if (nchunks >= 2) wait_chunk(nchunks - 2);
  if (nchunks >= 1) wait_chunk(nchunks - 1);
  tc_epilogue<C_GLOBAL>(s, M, N, C, ldc, scale);
}

}  // namespace fmm
