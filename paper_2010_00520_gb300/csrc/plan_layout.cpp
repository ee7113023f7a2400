// Layouts of the compressed formats, pointer binding and the host restore.
#include "plan_layout.h"

#include <algorithm>
#include <cmath>
#include <functional>

namespace fmm {

BufRef Layout::put(const cdouble* src, size_t count) {
  BufRef r;
  r.buf = 0;
  r.off = (int64_t)pack.size();
  pack.insert(pack.end(), src, src + count);
  return r;
}

BufRef Layout::scratch_alloc(int64_t count) {
  BufRef r;
  r.buf = 1;
  r.off = scratch;
  scratch += count;
  return r;
}

static BufRef offset(BufRef b, int64_t by) {
  b.off += by;
  return b;
}

static GemmSpec gemm(BufRef A, BufRef B, BufRef C, int M, int N, int K) {
  GemmSpec g;
  g.A = A;
  g.B = B;
  g.C = C;
  g.M = M;
  g.N = N;
  g.K = K;
  return g;
}

static void finish_ranks(Layout& L) {
  L.rmax_a = 0;
  L.rmax_b = 0;
  for (const auto& s : L.slabs) {
    L.rmax_a = std::max(L.rmax_a, s.ra);
    L.rmax_b = std::max(L.rmax_b, s.rb);
  }
}

// ---------------------------------------------------------------------------
// Tucker-3D (Fig. 3(a)): per direction C_p, U1_p, U2_p, U3_p.
// Pre-pass: H_p = U1_p . mat(C_p) (n1 x r2 r3).
// ---------------------------------------------------------------------------
void layout_tucker3d(const std::vector<Tucker3>& tk, const int n[3], Layout& L) {
  const int n_dir = (int)tk.size();
  L = Layout();
  for (int i = 0; i < 3; ++i) L.n[i] = n[i];
  L.n_dir = n_dir;
  L.yz_fmt = 1;
  L.stages.assign(1, {});
  L.ranks3.assign((size_t)n_dir * 3, 0);
  for (int p = 0; p < n_dir; ++p) {
    const Tucker3& t = tk[p];
    const int r1 = t.r[0], r2 = t.r[1], r3 = t.r[2];
    BufRef core = L.put(t.core), u1 = L.put(t.U[0]), u2 = L.put(t.U[1]), u3 = L.put(t.U[2]);
    BufRef h = L.scratch_alloc((int64_t)n[0] * r2 * r3);
    L.stages[0].push_back(gemm(u1, core, h, n[0], r2 * r3, r1));
    SlabSpec s;
    s.h = h;
    s.hx = (int64_t)r2 * r3;
    s.u2 = u2;
    s.u3 = u3;
    s.ra = r2;
    s.rb = r3;
    L.slabs.push_back(s);
    L.elements += (int64_t)t.core.size() + t.U[0].size() + t.U[1].size() + t.U[2].size();
    for (int i = 0; i < 3; ++i) {
      L.ranks3[(size_t)p * 3 + i] = t.r[i];
      L.rank[i] = std::max(L.rank[i], t.r[i]);
      L.mean_rank[i] += t.r[i] / (double)n_dir;
    }
  }
  finish_ranks(L);
}

// ---------------------------------------------------------------------------
// TT-3D (Fig. 4(a)): per direction U1_p, C1_p, U3_p.
// Pre-pass: T1_p = U1_p . mat(C1_p) (n1 x n2 r2); slab = T1_p[x] U3_p^T.
// ---------------------------------------------------------------------------
void layout_tt3d(const std::vector<TT3>& tt, const int n[3], Layout& L) {
  const int n_dir = (int)tt.size();
  L = Layout();
  for (int i = 0; i < 3; ++i) L.n[i] = n[i];
  L.n_dir = n_dir;
  L.yz_fmt = 2;
  L.stages.assign(1, {});
  L.ranks3.assign((size_t)n_dir * 3, 0);
  for (int p = 0; p < n_dir; ++p) {
    const TT3& t = tt[p];
    BufRef u1 = L.put(t.U1), c1 = L.put(t.C1), u3 = L.put(t.U3);
    BufRef t1 = L.scratch_alloc((int64_t)n[0] * n[1] * t.r2);
    L.stages[0].push_back(gemm(u1, c1, t1, n[0], n[1] * t.r2, t.r1));
    SlabSpec s;
    s.h = t1;
    s.hx = (int64_t)n[1] * t.r2;
    s.u3 = u3;
    s.ra = 0;
    s.rb = t.r2;
    L.slabs.push_back(s);
    L.elements += (int64_t)t.U1.size() + t.C1.size() + t.U3.size();
    const int r[2] = {t.r1, t.r2};
    for (int i = 0; i < 2; ++i) {
      L.ranks3[(size_t)p * 3 + i] = r[i];
      L.rank[i] = std::max(L.rank[i], r[i]);
      L.mean_rank[i] += r[i] / (double)n_dir;
    }
  }
  finish_ranks(L);
}

// ---------------------------------------------------------------------------
// Tucker-4D (Fig. 3(b)): C (r1 r2 r3 r4), U1..U4.
// Pre-pass: C_all = U4 . C^(4)T (n_dir x r1 r2 r3: row p = core of direction
// p), then H_p = U1 . mat(C_p).  Slab as Tucker-3D with the shared U2, U3.
// ---------------------------------------------------------------------------
void layout_tucker4d(const Tucker4& tk, const int n[3], int n_dir, Layout& L) {
  L = Layout();
  for (int i = 0; i < 3; ++i) L.n[i] = n[i];
  L.n_dir = n_dir;
  L.yz_fmt = 1;
  const int r1 = tk.r[0], r2 = tk.r[1], r3 = tk.r[2], r4 = tk.r[3];
  const int64_t R3 = (int64_t)r1 * r2 * r3;
  std::vector<cdouble> c4t((size_t)r4 * R3);
  for (int64_t abc = 0; abc < R3; ++abc)
    for (int d = 0; d < r4; ++d) c4t[(size_t)d * R3 + abc] = tk.core[(size_t)abc * r4 + d];
  BufRef u1 = L.put(tk.U[0]), u2 = L.put(tk.U[1]), u3 = L.put(tk.U[2]), u4 = L.put(tk.U[3]);
  BufRef ct = L.put(c4t);
  BufRef call = L.scratch_alloc((int64_t)n_dir * R3);
  BufRef h = L.scratch_alloc((int64_t)n_dir * n[0] * r2 * r3);
  L.stages.assign(2, {});
  L.stages[0].push_back(gemm(u4, ct, call, n_dir, (int)R3, r4));
  for (int p = 0; p < n_dir; ++p) {
    BufRef hp = offset(h, (int64_t)p * n[0] * r2 * r3);
    L.stages[1].push_back(gemm(u1, offset(call, p * R3), hp, n[0], r2 * r3, r1));
    SlabSpec s;
    s.h = hp;
    s.hx = (int64_t)r2 * r3;
    s.u2 = u2;
    s.u3 = u3;
    s.ra = r2;
    s.rb = r3;
    L.slabs.push_back(s);
  }
  L.elements = (int64_t)tk.core.size() + tk.U[0].size() + tk.U[1].size() + tk.U[2].size() + tk.U[3].size();
  for (int i = 0; i < 4; ++i) L.rank[i] = tk.r[i];
  for (int i = 0; i < 3; ++i) L.mean_rank[i] = tk.r[i];
  finish_ranks(L);
}

// ---------------------------------------------------------------------------
// H-Tucker (Fig. 3(c)): leaves U1..U4, C12 ((r1 r2) x r12), B (r12 x r34),
// C34 ((r3 r4) x r34), stored as C34p[l][t][c] = C34[c l][t].
// Pre-pass: E = C12 B; V = U4 . C34p (row p: V_p[t][c]); C_p = E V_p
// (r1 r2 x r3, the core of direction p); H_p = U1 . mat(C_p).
// ---------------------------------------------------------------------------
void layout_htucker(const HTucker4& ht, const int n[3], int n_dir, Layout& L) {
  L = Layout();
  for (int i = 0; i < 3; ++i) L.n[i] = n[i];
  L.n_dir = n_dir;
  L.yz_fmt = 1;
  const int r1 = ht.r[0], r2 = ht.r[1], r3 = ht.r[2], r4 = ht.r[3], r12 = ht.r[4], r34 = ht.r[5];
  std::vector<cdouble> c34p((size_t)r4 * r34 * r3);
  for (int c = 0; c < r3; ++c)
    for (int l = 0; l < r4; ++l)
      for (int t = 0; t < r34; ++t)
        c34p[((size_t)l * r34 + t) * r3 + c] = ht.C34[((size_t)c * r4 + l) * r34 + t];
  BufRef u1 = L.put(ht.U[0]), u2 = L.put(ht.U[1]), u3 = L.put(ht.U[2]), u4 = L.put(ht.U[3]);
  BufRef c12 = L.put(ht.C12), bm = L.put(ht.B), c34 = L.put(c34p);
  const int64_t R12 = (int64_t)r1 * r2;
  BufRef e = L.scratch_alloc(R12 * r34);
  BufRef v = L.scratch_alloc((int64_t)n_dir * r34 * r3);
  BufRef call = L.scratch_alloc((int64_t)n_dir * R12 * r3);
  BufRef h = L.scratch_alloc((int64_t)n_dir * n[0] * r2 * r3);
  L.stages.assign(3, {});
  L.stages[0].push_back(gemm(c12, bm, e, (int)R12, r34, r12));
  L.stages[0].push_back(gemm(u4, c34, v, n_dir, r34 * r3, r4));
  for (int p = 0; p < n_dir; ++p) {
    BufRef cp = offset(call, p * R12 * r3);
    BufRef hp = offset(h, (int64_t)p * n[0] * r2 * r3);
    L.stages[1].push_back(gemm(e, offset(v, (int64_t)p * r34 * r3), cp, (int)R12, r3, r34));
    L.stages[2].push_back(gemm(u1, cp, hp, n[0], r2 * r3, r1));
    SlabSpec s;
    s.h = hp;
    s.hx = (int64_t)r2 * r3;
    s.u2 = u2;
    s.u3 = u3;
    s.ra = r2;
    s.rb = r3;
    L.slabs.push_back(s);
  }
  L.elements = (int64_t)ht.U[0].size() + ht.U[1].size() + ht.U[2].size() + ht.U[3].size() + ht.C12.size() +
               ht.C34.size() + ht.B.size();
  for (int i = 0; i < 6; ++i) L.rank[i] = ht.r[i];
  for (int i = 0; i < 3; ++i) L.mean_rank[i] = ht.r[i];
  finish_ranks(L);
}

// ---------------------------------------------------------------------------
// TT-4D (Fig. 4(b)): U1 (n1 x r1), C1 (r1 x n2 x r2), C2 (r2 x n3 x r3), U3
// (n_dir x r3); C2 stored as C2p[t][z][b] = C2[b][z][t].
// Pre-pass: T1 = U1 . mat(C1) (shared by all directions) and R = U3 . C2p
// (row p: R_p[z][b] = S_p[b][z], the slice of Fig. 4(b)); slab = T1[x] R_p^T.
// ---------------------------------------------------------------------------
void layout_tt4d(const TT4& tt, const int n[3], int n_dir, Layout& L) {
  L = Layout();
  for (int i = 0; i < 3; ++i) L.n[i] = n[i];
  L.n_dir = n_dir;
  L.yz_fmt = 2;
  const int r1 = tt.r[0], r2 = tt.r[1], r3 = tt.r[2];
  std::vector<cdouble> c2p((size_t)r3 * n[2] * r2);
  for (int b = 0; b < r2; ++b)
    for (int z = 0; z < n[2]; ++z)
      for (int t = 0; t < r3; ++t) c2p[((size_t)t * n[2] + z) * r2 + b] = tt.C2[((size_t)b * n[2] + z) * r3 + t];
  BufRef u1 = L.put(tt.U1), c1 = L.put(tt.C1), c2 = L.put(c2p), u3 = L.put(tt.U3);
  BufRef t1 = L.scratch_alloc((int64_t)n[0] * n[1] * r2);
  BufRef rall = L.scratch_alloc((int64_t)n_dir * n[2] * r2);
  L.stages.assign(1, {});
  L.stages[0].push_back(gemm(u1, c1, t1, n[0], n[1] * r2, r1));
  L.stages[0].push_back(gemm(u3, c2, rall, n_dir, n[2] * r2, r3));
  for (int p = 0; p < n_dir; ++p) {
    SlabSpec s;
    s.h = t1;
    s.hx = (int64_t)n[1] * r2;
    s.u3 = offset(rall, (int64_t)p * n[2] * r2);
    s.ra = 0;
    s.rb = r2;
    L.slabs.push_back(s);
  }
  L.elements = (int64_t)tt.U1.size() + tt.C1.size() + tt.C2.size() + tt.U3.size();
  for (int i = 0; i < 3; ++i) {
    L.rank[i] = tt.r[i];
    L.mean_rank[i] = tt.r[i];
  }
  finish_ranks(L);
}

// ---------------------------------------------------------------------------
// binding
// ---------------------------------------------------------------------------
static const void* cptr(BufRef b, const void* pack, void* scratch, size_t es) {
  const char* base = b.buf == 0 ? (const char*)pack : (const char*)scratch;
  return base + (size_t)b.off * es;
}

void bind_gemms(const Layout& L, const void* pack, void* scratch, size_t es,
                std::vector<std::vector<GemmDesc>>& out) {
  out.assign(L.stages.size(), {});
  for (size_t s = 0; s < L.stages.size(); ++s)
    for (const GemmSpec& g : L.stages[s]) {
      GemmDesc d;
      d.A = cptr(g.A, pack, scratch, es);
      d.B = cptr(g.B, pack, scratch, es);
      d.C = const_cast<void*>(cptr(g.C, pack, scratch, es));
      d.M = g.M;
      d.N = g.N;
      d.K = g.K;
      d.pad = 0;
      out[s].push_back(d);
    }
}

void bind_slabs(const Layout& L, const void* pack, void* scratch, size_t es, std::vector<SlabDesc>& out) {
  out.clear();
  for (const SlabSpec& s : L.slabs) {
    SlabDesc d;
    d.h = cptr(s.h, pack, scratch, es);
    d.u2 = s.ra > 0 ? cptr(s.u2, pack, scratch, es) : nullptr;
    d.u3 = cptr(s.u3, pack, scratch, es);
    d.hx = s.hx;
    d.ra = s.ra;
    d.rb = s.rb;
    out.push_back(d);
  }
}

// ---------------------------------------------------------------------------
// host restore (FP64)
// ---------------------------------------------------------------------------
namespace {

// The pre-pass products of a layout, run on the host into `scratch`.
void host_prepass(const Layout& L, std::vector<cdouble>& scratch) {
  scratch.assign((size_t)std::max<int64_t>(L.scratch, 1), cdouble(0.0, 0.0));
  std::vector<std::vector<GemmDesc>> st;
  bind_gemms(L, L.pack.data(), scratch.data(), sizeof(cdouble), st);
  for (const auto& stage : st)
    parallel_for((int)stage.size(), [&](int i) {
      const GemmDesc& g = stage[i];
      const cdouble* A = (const cdouble*)g.A;
      const cdouble* B = (const cdouble*)g.B;
      cdouble* C = (cdouble*)g.C;
      // row m of C accumulates A[m][k] B[k][:] in the order of k
      for (int m = 0; m < g.M; ++m) {
        cdouble* c = C + (size_t)m * g.N;
        for (int nn = 0; nn < g.N; ++nn) c[nn] = cdouble(0.0, 0.0);
        for (int k = 0; k < g.K; ++k) caxpy(A[(size_t)m * g.K + k], B + (size_t)k * g.N, c, (size_t)g.N);
      }
    });
}

// Direction p's slab formula for every x: o = T~_p[x][y][z] (n1 x n2 x n3).
void host_slabs(const Layout& L, const SlabDesc& d, cdouble* o) {
  const int n1 = L.n[0], n2 = L.n[1], n3 = L.n[2];
  const cdouble* U3 = (const cdouble*)d.u3;
  std::vector<cdouble> G((size_t)n2 * d.rb);
  for (int x = 0; x < n1; ++x) {
    const cdouble* H = (const cdouble*)d.h + (size_t)x * d.hx;
    if (L.yz_fmt == 1) {
      const cdouble* U2 = (const cdouble*)d.u2;
      for (int y = 0; y < n2; ++y) {
        cdouble* g = &G[(size_t)y * d.rb];
        for (int c = 0; c < d.rb; ++c) g[c] = cdouble(0.0, 0.0);
        for (int b = 0; b < d.ra; ++b) caxpy(U2[(size_t)y * d.ra + b], H + (size_t)b * d.rb, g, (size_t)d.rb);
      }
    } else {
      for (size_t i = 0; i < (size_t)n2 * d.rb; ++i) G[i] = H[i];
    }
    cdouble* ox = o + (size_t)x * n2 * n3;
    for (int y = 0; y < n2; ++y)
      for (int z = 0; z < n3; ++z) ox[(size_t)y * n3 + z] = cdot(U3 + (size_t)z * d.rb, &G[(size_t)y * d.rb], d.rb);
  }
}

}  // namespace

void restore_host(const Layout& L, std::vector<cdouble>& out) {
  std::vector<cdouble> scratch;
  host_prepass(L, scratch);
  std::vector<SlabDesc> sl;
  bind_slabs(L, L.pack.data(), scratch.data(), sizeof(cdouble), sl);
  const size_t per = (size_t)L.n[0] * L.n[1] * L.n[2];
  out.assign(per * L.n_dir, cdouble(0.0, 0.0));
  parallel_for(L.n_dir, [&](int p) { host_slabs(L, sl[p], &out[per * p]); });
}

double restore_error_host(const Layout& L, const std::function<void(int, std::vector<cdouble>&)>& op) {
  std::vector<cdouble> scratch;
  host_prepass(L, scratch);
  std::vector<SlabDesc> sl;
  bind_slabs(L, L.pack.data(), scratch.data(), sizeof(cdouble), sl);
  const size_t per = (size_t)L.n[0] * L.n[1] * L.n[2];
  // per-direction sums, added in direction order: the result does not depend
  // on how the directions were spread over the threads
  std::vector<double> diff2(L.n_dir, 0.0), norm2(L.n_dir, 0.0);
  parallel_for(L.n_dir, [&](int p) {
    std::vector<cdouble> T, R(per);
    op(p, T);
    host_slabs(L, sl[p], R.data());
    double e = 0.0, t = 0.0;
    for (size_t i = 0; i < per; ++i) {
      e += std::norm(T[i] - R[i]);
      t += std::norm(T[i]);
    }
    diff2[p] = e;
    norm2[p] = t;
  });
  double e = 0.0, t = 0.0;
  for (int p = 0; p < L.n_dir; ++p) {
    e += diff2[p];
    t += norm2[p];
  }
  return t > 0.0 ? std::sqrt(e / t) : 0.0;
}

}  // namespace fmm
