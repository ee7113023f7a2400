// FP64 host decompositions: TT-SVD per direction and the 4D formats.
#include "host_decomp.h"

#include <algorithm>
#include <cmath>

namespace fmm {

// ---------------------------------------------------------------------------
// Hermitian eigen-decomposition: Householder tridiagonalisation + QL
// ---------------------------------------------------------------------------

// Implicit-shift QL iterations on the real symmetric tridiagonal matrix with
// diagonal d[0..n) and off-diagonal e[i] = T[i+1][i] (e[n-1] unused), the
// published method of Bowdler, Martin, Reinsch and Wilkinson ("The QR and QL
// algorithms for symmetric matrices", Numer. Math. 11, 1968): Wilkinson-type
// shift from the trailing 2 x 2 block, a chain of plane rotations per sweep; the
// rotations are accumulated into the eigenvector matrix, stored transposed
// (Zt[j] is eigenvector j, contiguous) so that a rotation of two vectors
// touches two contiguous rows.  The rotations of one iteration are recorded
// and then applied to blocks of columns of Zt on the host cores: every
// column sees the same rotations in the same order as one at a time would
// apply them, so the result does not depend on the split.
static void tridiag_ql(int n, std::vector<double>& d, std::vector<double>& e, std::vector<double>& Zt) {
  const double eps = 2.220446049250313e-16;
  e.resize(n);
  e[n - 1] = 0.0;
  std::vector<double> rc(n), rs(n);
  // rotations i = hi, hi - 1, ..., lo of rows (i, i + 1)
  auto rotate = [&](int hi, int lo) {
    if (hi < lo) return;
    constexpr int kCols = 64;
    auto block = [&](int b) {
      const int k0 = b * kCols, k1 = std::min(n, k0 + kCols);
      for (int i = hi; i >= lo; --i) {
        const double c = rc[i], s = rs[i];
        double* za = &Zt[(size_t)i * n];
        double* zb = &Zt[(size_t)(i + 1) * n];
        for (int k = k0; k < k1; ++k) {
          const double zi = za[k], zi1 = zb[k];
          zb[k] = s * zi + c * zi1;
          za[k] = c * zi - s * zi1;
        }
      }
    };
    const int nb = (n + kCols - 1) / kCols;
    if ((int64_t)(hi - lo + 1) * n >= (1 << 16) && nb > 1) {
      parallel_for(nb, block);
    } else {
      for (int b = 0; b < nb; ++b) block(b);
    }
  };
  for (int l = 0; l < n; ++l) {
    for (int iter = 0; iter < 100; ++iter) {
      int m = l;
      for (; m < n - 1; ++m) {
        const double dd = std::fabs(d[m]) + std::fabs(d[m + 1]);
        if (std::fabs(e[m]) <= eps * dd) break;
      }
      if (m == l) break;
      // Wilkinson-type shift from the leading 2 x 2 block at l
      double g = (d[l + 1] - d[l]) / (2.0 * e[l]);
      double r = std::hypot(g, 1.0);
      g = d[m] - d[l] + e[l] / (g + (g >= 0 ? r : -r));
      double s = 1.0, c = 1.0, p = 0.0;
      int i = m - 1;
      bool underflow = false;
      for (; i >= l; --i) {
        const double f = s * e[i], b = c * e[i];
        r = std::hypot(f, g);
        e[i + 1] = r;
        if (r == 0.0) {
          d[i + 1] -= p;
          e[m] = 0.0;
          underflow = true;
          break;
        }
        s = f / r;
        c = g / r;
        g = d[i + 1] - p;
        r = (d[i] - g) * s + 2.0 * c * b;
        p = s * r;
        d[i + 1] = g + p;
        g = c * r - b;
        rc[i] = c;
        rs[i] = s;
      }
      // recorded: m - 1 down to l, or down to i + 1 when the sweep stopped early
      rotate(m - 1, underflow ? i + 1 : l);
      if (underflow) continue;
      d[l] -= p;
      e[l] = g;
      e[m] = 0.0;
    }
  }
}

void hermitian_eig_tridiag(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V) {
  std::vector<cdouble> Q((size_t)n * n, cdouble(0.0, 0.0));
  for (int i = 0; i < n; ++i) Q[(size_t)i * n + i] = 1.0;
  std::vector<cdouble> v(n), p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;               // length of the column below the diagonal
    double xn2 = 0.0;
    for (int i = 0; i < m; ++i) xn2 += std::norm(A[(size_t)(k + 1 + i) * n + k]);
    const double xnorm = std::sqrt(xn2);
    if (xnorm == 0.0) continue;
    const cdouble x0 = A[(size_t)(k + 1) * n + k];
    const cdouble phase = std::abs(x0) > 0.0 ? x0 / std::abs(x0) : cdouble(1.0, 0.0);
    const cdouble alpha = -phase * xnorm;
    for (int i = 0; i < m; ++i) v[i] = A[(size_t)(k + 1 + i) * n + k];
    v[0] -= alpha;
    double vn2 = 0.0;
    for (int i = 0; i < m; ++i) vn2 += std::norm(v[i]);
    if (vn2 == 0.0) continue;
    const double inv = 1.0 / std::sqrt(vn2);
    for (int i = 0; i < m; ++i) v[i] *= inv;
    // p = A_sub v, beta = v^H p, w = 2 (p - beta v); A_sub -= v w^H + w v^H
    parallel_for(m, [&](int i) { p[i] = cdot(&A[(size_t)(k + 1 + i) * n + k + 1], v.data(), m); });
    double beta = 0.0;
    for (int i = 0; i < m; ++i) beta += (std::conj(v[i]) * p[i]).real();
    for (int i = 0; i < m; ++i) w[i] = 2.0 * (p[i] - beta * v[i]);
    parallel_for(m, [&](int i) {
      cdouble* row = &A[(size_t)(k + 1 + i) * n + k + 1];
      caxpy_conj(-v[i], w.data(), row, m);
      caxpy_conj(-w[i], v.data(), row, m);
    });
    for (int i = 0; i < m; ++i) {
      A[(size_t)(k + 1 + i) * n + k] = (i == 0) ? alpha : cdouble(0.0, 0.0);
      A[(size_t)k * n + k + 1 + i] = (i == 0) ? std::conj(alpha) : cdouble(0.0, 0.0);
    }
    // Q <- Q H_k, H_k = I - 2 v v^H on indices k+1 .. n-1
    parallel_for(n, [&](int r) {
      cdouble* q = &Q[(size_t)r * n + k + 1];
      caxpy_conj(-2.0 * cdot(q, v.data(), m), v.data(), q, m);
    });
  }
  // T = D T' D^H with T' real: phases make every off-diagonal |e_k|
  std::vector<double> d(n), e(n, 0.0);
  std::vector<cdouble> ph(n, cdouble(1.0, 0.0));
  for (int k = 0; k < n; ++k) d[k] = A[(size_t)k * n + k].real();
  for (int k = 0; k + 1 < n; ++k) {
    const cdouble ek = A[(size_t)(k + 1) * n + k];
    const double a = std::abs(ek);
    e[k] = a;
    ph[k + 1] = a > 0.0 ? ph[k] * (ek / a) : ph[k];
  }
  std::vector<double> Zt((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Zt[(size_t)i * n + i] = 1.0;
  tridiag_ql(n, d, e, Zt);
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int i, int j) { return d[i] > d[j]; });
  lam.assign(n, 0.0);
  for (int c = 0; c < n; ++c) lam[c] = d[idx[c]];
  // V = Q D Z (columns reordered); Z[j][col] = Zt[col][j]
  V.assign((size_t)n * n, cdouble(0.0, 0.0));
  parallel_for(n, [&](int r) {
    const cdouble* q = &Q[(size_t)r * n];
    cdouble* out = &V[(size_t)r * n];
    std::vector<cdouble> qd(n);
    for (int j = 0; j < n; ++j) qd[j] = q[j] * ph[j];
    for (int c = 0; c < n; ++c) {
      const double* z = &Zt[(size_t)idx[c] * n];
      cdouble acc(0.0, 0.0);
      for (int j = 0; j < n; ++j) acc += qd[j] * z[j];
      out[c] = acc;
    }
  });
}

void hermitian_eig_auto(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V) {
  if (n <= 96) hermitian_eig(n, A, lam, V);
  else hermitian_eig_tridiag(n, A, lam, V);
}

double step_budget(double normT, double gamma, double parts, int rule) {
  return rule == 0 ? gamma * normT / std::sqrt(parts) : gamma / std::sqrt(parts);
}

// ---------------------------------------------------------------------------
// truncated left singular basis through the smaller Gram matrix
// ---------------------------------------------------------------------------
int truncated_left(const cdouble* A, int64_t m, int64_t N, double delta, int rule,
                   std::vector<cdouble>& U, std::vector<cdouble>& Q) {
  std::vector<double> lam;
  std::vector<cdouble> V;
  int r;
  if (m <= N) {
    // G = A A^H (m x m)
    std::vector<cdouble> G((size_t)m * m, cdouble(0.0, 0.0));
    std::vector<const cdouble*> rows(m);
    for (int64_t i = 0; i < m; ++i) rows[i] = A + (size_t)i * N;
    gram_upper(rows.data(), m, N, G.data());
    for (int64_t i = 0; i < m; ++i)
      for (int64_t j = i + 1; j < m; ++j) G[(size_t)j * m + i] = std::conj(G[(size_t)i * m + j]);
    hermitian_eig_auto((int)m, G, lam, V);
    r = truncation_rank(lam, delta, rule);
    U.assign((size_t)m * r, cdouble(0.0, 0.0));
    for (int64_t i = 0; i < m; ++i)
      for (int c = 0; c < r; ++c) U[(size_t)i * r + c] = V[(size_t)i * m + c];
  } else {
    // G = A^H A (N x N): G[i][j] = sum_row conj(A[row][i]) A[row][j]
    std::vector<cdouble> G((size_t)N * N, cdouble(0.0, 0.0));
    // G = conj(At At^H) with At = A^T (N x m): the Gram of At's rows
    std::vector<cdouble> At((size_t)N * m);
    parallel_for((int)N, [&](int i) {
      for (int64_t row = 0; row < m; ++row) At[(size_t)i * m + row] = A[(size_t)row * N + i];
    });
    std::vector<const cdouble*> rows(N);
    for (int64_t i = 0; i < N; ++i) rows[i] = &At[(size_t)i * m];
    gram_upper(rows.data(), N, m, G.data());
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = i; j < N; ++j) G[(size_t)i * N + j] = std::conj(G[(size_t)i * N + j]);
    for (int64_t i = 0; i < N; ++i)
      for (int64_t j = i + 1; j < N; ++j) G[(size_t)j * N + i] = std::conj(G[(size_t)i * N + j]);
    hermitian_eig_auto((int)N, G, lam, V);
    r = truncation_rank(lam, delta, rule);
    // keep only directions with a usable singular value
    const double floor = std::max(lam[0], 0.0) * 1e-28;
    while (r > 1 && !(lam[r - 1] > floor)) --r;
    // U = A V_r Sigma_r^-1
    U.assign((size_t)m * r, cdouble(0.0, 0.0));
    std::vector<double> isig(r);
    for (int c = 0; c < r; ++c) isig[c] = lam[c] > 0.0 ? 1.0 / std::sqrt(lam[c]) : 0.0;
    parallel_for((int)m, [&](int row) {
      const cdouble* a = A + (size_t)row * N;
      cdouble* u = &U[(size_t)row * r];
      for (int64_t k = 0; k < N; ++k) caxpy(a[k], &V[(size_t)k * N], u, (size_t)r);
      for (int c = 0; c < r; ++c) u[c] *= isig[c];
    });
  }
  // Q = U^H A (r x N)
  Q.assign((size_t)r * N, cdouble(0.0, 0.0));
  parallel_for(r, [&](int c) {
    cdouble* q = &Q[(size_t)c * N];
    for (int64_t row = 0; row < m; ++row) caxpy(std::conj(U[(size_t)row * r + c]), A + (size_t)row * N, q, (size_t)N);
  });
  return r;
}

// ---------------------------------------------------------------------------
// TT-SVD of one direction (3D format)
// ---------------------------------------------------------------------------
void ttsvd3(const std::vector<cdouble>& T, const int n[3], double gamma, int rule, TT3& out) {
  const int n1 = n[0], n2 = n[1], n3 = n[2];
  double norm2 = 0.0;
  for (auto& z : T) norm2 += std::norm(z);
  const double delta = step_budget(std::sqrt(norm2), gamma, 2.0, rule);
  std::vector<cdouble> Q1, U2, Q2;
  out.r1 = truncated_left(T.data(), n1, (int64_t)n2 * n3, delta, rule, out.U1, Q1);
  // Q1 (r1 x n2 n3) as (r1 n2) x n3
  out.r2 = truncated_left(Q1.data(), (int64_t)out.r1 * n2, n3, delta, rule, out.C1, Q2);
  // U3[z][b] = Q2[b][z]
  out.U3.assign((size_t)n3 * out.r2, cdouble(0.0, 0.0));
  for (int b = 0; b < out.r2; ++b)
    for (int z = 0; z < n3; ++z) out.U3[(size_t)z * out.r2 + b] = Q2[(size_t)b * n3 + z];
}

// ---------------------------------------------------------------------------
// Tucker of T_4D (HOSVD, Alg. 1)
// ---------------------------------------------------------------------------
void hosvd4(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double delta, int rule, Tucker4& out) {
  const int n1 = n[0], n2 = n[1], n3 = n[2];
  const int K = (int)Tp.size();
  const size_t N = (size_t)n1 * n2 * n3;
  // modal Gram matrices of modes 1..3: sums of the per-direction ones
  std::vector<std::vector<cdouble>> g1(K), g2(K), g3(K);
  parallel_for(K, [&](int p) {
    const cdouble* T = Tp[p].data();
    g1[p].assign((size_t)n1 * n1, cdouble(0.0, 0.0));
    g2[p].assign((size_t)n2 * n2, cdouble(0.0, 0.0));
    g3[p].assign((size_t)n3 * n3, cdouble(0.0, 0.0));
    const size_t len = (size_t)n2 * n3;
    for (int i = 0; i < n1; ++i)
      for (int j = i; j < n1; ++j) g1[p][(size_t)i * n1 + j] = cdot_conj(T + i * len, T + j * len, len);
    for (int x = 0; x < n1; ++x) {
      const cdouble* S = T + (size_t)x * len;
      for (int i = 0; i < n2; ++i)
        for (int j = i; j < n2; ++j) g2[p][(size_t)i * n2 + j] += cdot_conj(S + (size_t)i * n3, S + (size_t)j * n3, n3);
    }
    for (size_t row = 0; row < (size_t)n1 * n2; ++row) {
      const cdouble* v = T + row * n3;
      for (int i = 0; i < n3; ++i) caxpy_conj(v[i], v + i, &g3[p][(size_t)i * n3 + i], n3 - i);
    }
  });
  std::vector<cdouble> G[4];
  const int dims[4] = {n1, n2, n3, K};
  for (int mode = 0; mode < 3; ++mode) {
    const int m = dims[mode];
    auto& src = mode == 0 ? g1 : (mode == 1 ? g2 : g3);
    G[mode].assign((size_t)m * m, cdouble(0.0, 0.0));
    for (int p = 0; p < K; ++p)
      for (size_t i = 0; i < (size_t)m * m; ++i) G[mode][i] += src[p][i];
  }
  // mode 4: G4[p][q] = <T_p, T_q>
  G[3].assign((size_t)K * K, cdouble(0.0, 0.0));
  {
    std::vector<const cdouble*> rows(K);
    for (int p = 0; p < K; ++p) rows[p] = Tp[p].data();
    gram_upper(rows.data(), K, (int64_t)N, G[3].data());
  }
  for (int mode = 0; mode < 4; ++mode) {
    const int m = dims[mode];
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) G[mode][(size_t)j * m + i] = std::conj(G[mode][(size_t)i * m + j]);
    std::vector<double> lam;
    std::vector<cdouble> V;
    hermitian_eig_auto(m, G[mode], lam, V);
    const int r = truncation_rank(lam, delta, rule);
    out.r[mode] = r;
    out.U[mode].assign((size_t)m * r, cdouble(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < r; ++c) out.U[mode][(size_t)i * r + c] = V[(size_t)i * m + c];
  }
  const int r1 = out.r[0], r2 = out.r[1], r3 = out.r[2], r4 = out.r[3];
  const size_t R3 = (size_t)r1 * r2 * r3;
  // per-direction projection Y_p = T_p x1 U1^H x2 U2^H x3 U3^H (U3^H stored
  // row by row so that the last sum runs over contiguous memory)
  std::vector<cdouble> U3h((size_t)r3 * n3);
  for (int z = 0; z < n3; ++z)
    for (int c = 0; c < r3; ++c) U3h[(size_t)c * n3 + z] = std::conj(out.U[2][(size_t)z * r3 + c]);
  std::vector<std::vector<cdouble>> Y(K);
  parallel_for(K, [&](int p) {
    const cdouble* T = Tp[p].data();
    const size_t len = (size_t)n2 * n3;
    std::vector<cdouble> Y1((size_t)r1 * len, cdouble(0.0, 0.0));
    for (int x = 0; x < n1; ++x)
      for (int a = 0; a < r1; ++a) caxpy(std::conj(out.U[0][(size_t)x * r1 + a]), T + x * len, &Y1[a * len], len);
    std::vector<cdouble> Y2((size_t)r1 * r2 * n3, cdouble(0.0, 0.0));
    for (int a = 0; a < r1; ++a)
      for (int y = 0; y < n2; ++y)
        for (int b = 0; b < r2; ++b)
          caxpy(std::conj(out.U[1][(size_t)y * r2 + b]), &Y1[((size_t)a * n2 + y) * n3], &Y2[((size_t)a * r2 + b) * n3],
                n3);
    Y[p].assign(R3, cdouble(0.0, 0.0));
    for (size_t ab = 0; ab < (size_t)r1 * r2; ++ab)
      for (int c = 0; c < r3; ++c) Y[p][ab * r3 + c] = cdot(&U3h[(size_t)c * n3], &Y2[ab * n3], n3);
  });
  // core[abc][d] = sum_p Y_p[abc] conj(U4[p][d])
  out.core.assign(R3 * r4, cdouble(0.0, 0.0));
  parallel_for((int)r1, [&](int a) {
    for (size_t bc = 0; bc < (size_t)r2 * r3; ++bc) {
      const size_t abc = (size_t)a * r2 * r3 + bc;
      cdouble* dst = &out.core[abc * r4];
      for (int p = 0; p < K; ++p) caxpy_conj(Y[p][abc], &out.U[3][(size_t)p * r4], dst, r4);
    }
  });
}

static double norm2_all(const std::vector<std::vector<cdouble>>& Tp) {
  double s = 0.0;
  for (auto& T : Tp)
    for (auto& z : T) s += std::norm(z);
  return s;
}

// ---------------------------------------------------------------------------
// H-Tucker (Alg. 2)
// ---------------------------------------------------------------------------
void htucker4(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double gamma, int rule, HTucker4& out) {
  const double delta = step_budget(std::sqrt(norm2_all(Tp)), gamma, 6.0, rule);
  Tucker4 tk;
  hosvd4(Tp, n, delta, rule, tk);
  for (int i = 0; i < 4; ++i) {
    out.r[i] = tk.r[i];
    out.U[i] = tk.U[i];
  }
  const int r1 = tk.r[0], r2 = tk.r[1], r3 = tk.r[2], r4 = tk.r[3];
  const int64_t m12 = (int64_t)r1 * r2, m34 = (int64_t)r3 * r4;
  // W12 = core as (r1 r2) x (r3 r4); node {1,2}: W12 ~ C12 S V^H, Q12 = S V^H
  std::vector<cdouble> Q12;
  out.r[4] = truncated_left(tk.core.data(), m12, m34, delta, rule, out.C12, Q12);
  const int r12 = out.r[4];
  // node {3,4}: its matricization W12^T = conj(V) S C12^T has the same
  // singular values, so the same rank at the same budget, and left singular
  // vectors conj(V) = (S^-1 Q12)^T; S is read off the row norms of Q12.
  // Directions whose singular value is lost in rounding are dropped, as in
  // the Gram route of truncated_left.
  std::vector<double> sig(r12, 0.0);
  parallel_for(r12, [&](int t) {
    double s2 = 0.0;
    for (int64_t j = 0; j < m34; ++j) s2 += std::norm(Q12[(size_t)t * m34 + j]);
    sig[t] = std::sqrt(s2);
  });
  int r34 = r12;
  while (r34 > 1 && !(sig[r34 - 1] > sig[0] * 1e-14)) --r34;
  out.r[5] = r34;
  out.C34.assign((size_t)m34 * r34, cdouble(0.0, 0.0));
  for (int t = 0; t < r34; ++t) {
    const double inv = 1.0 / sig[t];
    for (int64_t j = 0; j < m34; ++j) out.C34[(size_t)j * r34 + t] = Q12[(size_t)t * m34 + j] * inv;
  }
  // B = C12^H W12 conj(C34) = Q12 conj(C34)
  out.B.assign((size_t)r12 * r34, cdouble(0.0, 0.0));
  parallel_for(r12, [&](int s) {
    for (int t = 0; t < r34; ++t) {
      cdouble acc(0.0, 0.0);
      for (int64_t j = 0; j < m34; ++j) acc += Q12[(size_t)s * m34 + j] * std::conj(out.C34[(size_t)j * r34 + t]);
      out.B[(size_t)s * r34 + t] = acc;
    }
  });
}

// ---------------------------------------------------------------------------
// TT of T_4D through its Tucker core
// ---------------------------------------------------------------------------
void tt4_via_tucker(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double gamma, int rule, TT4& out) {
  const int n1 = n[0], n2 = n[1], n3 = n[2];
  const int K = (int)Tp.size();
  const double delta = step_budget(std::sqrt(norm2_all(Tp)), gamma, 7.0, rule);
  Tucker4 tk;
  hosvd4(Tp, n, delta, rule, tk);
  const int r1 = tk.r[0], r2 = tk.r[1], r3 = tk.r[2], r4 = tk.r[3];
  // TT-SVD of the core W (r1 x r2 x r3 x r4)
  std::vector<cdouble> G1, Q1, G2, Q2, G3, Q3;
  const int s1 = truncated_left(tk.core.data(), r1, (int64_t)r2 * r3 * r4, delta, rule, G1, Q1);
  const int s2 = truncated_left(Q1.data(), (int64_t)s1 * r2, (int64_t)r3 * r4, delta, rule, G2, Q2);
  const int s3 = truncated_left(Q2.data(), (int64_t)s2 * r3, r4, delta, rule, G3, Q3);
  out.r[0] = s1;
  out.r[1] = s2;
  out.r[2] = s3;
  // U1_TT = U1 G1 (n1 x s1)
  out.U1.assign((size_t)n1 * s1, cdouble(0.0, 0.0));
  for (int x = 0; x < n1; ++x)
    for (int a = 0; a < r1; ++a) {
      const cdouble u = tk.U[0][(size_t)x * r1 + a];
      for (int i = 0; i < s1; ++i) out.U1[(size_t)x * s1 + i] += u * G1[(size_t)a * s1 + i];
    }
  // C1[i][y][j] = sum_b G2[i][b][j] U2[y][b]
  out.C1.assign((size_t)s1 * n2 * s2, cdouble(0.0, 0.0));
  for (int i = 0; i < s1; ++i)
    for (int y = 0; y < n2; ++y)
      for (int b = 0; b < r2; ++b) {
        const cdouble u = tk.U[1][(size_t)y * r2 + b];
        const cdouble* g = &G2[((size_t)i * r2 + b) * s2];
        cdouble* dst = &out.C1[((size_t)i * n2 + y) * s2];
        for (int j = 0; j < s2; ++j) dst[j] += u * g[j];
      }
  // C2[j][z][k] = sum_c G3[j][c][k] U3[z][c]
  out.C2.assign((size_t)s2 * n3 * s3, cdouble(0.0, 0.0));
  for (int j = 0; j < s2; ++j)
    for (int z = 0; z < n3; ++z)
      for (int c = 0; c < r3; ++c) {
        const cdouble u = tk.U[2][(size_t)z * r3 + c];
        const cdouble* g = &G3[((size_t)j * r3 + c) * s3];
        cdouble* dst = &out.C2[((size_t)j * n3 + z) * s3];
        for (int k = 0; k < s3; ++k) dst[k] += u * g[k];
      }
  // U3_TT[p][k] = sum_d Q3[k][d] U4[p][d]
  out.U3.assign((size_t)K * s3, cdouble(0.0, 0.0));
  for (int p = 0; p < K; ++p)
    for (int k = 0; k < s3; ++k) {
      cdouble acc(0.0, 0.0);
      for (int d = 0; d < r4; ++d) acc += Q3[(size_t)k * r4 + d] * tk.U[3][(size_t)p * r4 + d];
      out.U3[(size_t)p * s3 + k] = acc;
    }
}

}  // namespace fmm
