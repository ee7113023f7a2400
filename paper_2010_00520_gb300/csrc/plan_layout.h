// Storage layout of the compressed formats and the restore schedule that goes
// with it.  A Layout holds the stored factors ("pack"), the size of the
// per-call restore scratch, the pre-pass products (GemmSpec, by stage) and the
// per-direction slab descriptors (SlabSpec), all addressed as (buffer,
// offset) pairs.  bind_* turns them into GemmDesc / SlabDesc for given base
// pointers: device pointers for the kernels, host pointers for the FP64 host
// interpreter (restore_host), which the set-up tests use to check every
// format's schedule on the CPU.
#pragma once

#include <cstdint>
#include <functional>
#include <vector>

#include "host_decomp.h"
#include "plan_internal.h"

namespace fmm {

struct BufRef {
  int buf = 0;          // 0: pack, 1: scratch
  int64_t off = 0;      // complex elements
};

struct GemmSpec {
  BufRef A, B, C;
  int M = 0, N = 0, K = 0;
};

struct SlabSpec {
  BufRef h, u2, u3;
  int64_t hx = 0;
  int ra = 0, rb = 0;
};

struct Layout {
  int n[3] = {0, 0, 0};
  int n_dir = 0;
  int yz_fmt = 1;                     // 1 Tucker-like, 2 TT-like
  std::vector<cdouble> pack;          // stored factors, in upload order
  int64_t scratch = 0;                // complex elements of restore scratch
  std::vector<std::vector<GemmSpec>> stages;
  std::vector<SlabSpec> slabs;        // n_dir entries
  int64_t elements = 0;               // stored elements (memory accounting)
  int rank[6] = {0, 0, 0, 0, 0, 0};   // largest ranks (see fmmfft_stats)
  double mean_rank[3] = {0, 0, 0};
  std::vector<int> ranks3;            // 3D formats: n_dir x 3 (TT-3D: r1, r2, 0)
  int rmax_a = 0, rmax_b = 0;

  BufRef put(const cdouble* src, size_t count);
  BufRef put(const std::vector<cdouble>& v) { return put(v.data(), v.size()); }
  BufRef scratch_alloc(int64_t count);
};

// Builders, one per format (the factor arrays' layouts are those of the
// structs in host_setup.h / host_decomp.h).
void layout_tucker3d(const std::vector<Tucker3>& tk, const int n[3], Layout& L);
void layout_tt3d(const std::vector<TT3>& tt, const int n[3], Layout& L);
void layout_tucker4d(const Tucker4& tk, const int n[3], int n_dir, Layout& L);
void layout_htucker(const HTucker4& ht, const int n[3], int n_dir, Layout& L);
void layout_tt4d(const TT4& tt, const int n[3], int n_dir, Layout& L);

// Pointer binding.  es: bytes per complex element of the bound buffers.
void bind_gemms(const Layout& L, const void* pack, void* scratch, size_t es,
                std::vector<std::vector<GemmDesc>>& out);
void bind_slabs(const Layout& L, const void* pack, void* scratch, size_t es, std::vector<SlabDesc>& out);

// FP64 host restoration of every direction from a layout (runs the pre-pass
// products and the slab formulas on the host).  out: n_dir x n1 x n2 x n3,
// T~_p[x][y][z] (unscaled).
void restore_host(const Layout& L, std::vector<cdouble>& out);

// FP64 relative error of the layout's restoration, sqrt(sum_p ||T~_p - R_p||^2
// / sum_p ||T~_p||^2) over all directions, where op(p, T) writes direction p's
// uncompressed T~_p (n1 x n2 x n3, same indexing as restore_host) and R_p is
// restored as in restore_host, one direction at a time.
double restore_error_host(const Layout& L, const std::function<void(int, std::vector<cdouble>&)>& op);

}  // namespace fmm
