// FP64 host set-up: directions, operator of Eq. 7, embedding + FFT, HOSVD.
#include "host_setup.h"
#include "host_decomp.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>

namespace fmm {

static const double kPiD = 3.14159265358979323846264338327950288;

// Set inside the worker threads: a parallel_for nested in another runs
// serially on the calling worker instead of spawning more threads.
static thread_local bool t_in_worker = false;

void parallel_for(int n, const std::function<void(int)>& fn) {
  if (n <= 0) return;
  unsigned hw = std::thread::hardware_concurrency();
  int nt = (int)std::min<unsigned>(hw ? hw : 1, (unsigned)n);
  if (nt <= 1 || t_in_worker) {
    for (int i = 0; i < n; ++i) fn(i);
    return;
  }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&]() {
      t_in_worker = true;
      for (int i = next.fetch_add(1); i < n; i = next.fetch_add(1)) fn(i);
    });
  for (auto& t : th) t.join();
}

void gram_upper(const cdouble* const* rows, int64_t m, int64_t N, cdouble* G) {
  constexpr int kB = 8;          // rows per block
  constexpr int64_t kC = 256;    // terms of the sum per chunk (4 KB of a row)
  const int64_t nb = (m + kB - 1) / kB;
  parallel_for((int)nb, [&](int b) {
    const int64_t i0 = (int64_t)b * kB;
    const int ni = (int)std::min<int64_t>(kB, m - i0);
    // partial sums [j - i0][u] (re, im) of block row u against row j
    std::vector<double> acc((size_t)(m - i0) * kB * 2, 0.0);
    for (int64_t k0 = 0; k0 < N; k0 += kC) {
      const int64_t kn = std::min(kC, N - k0);
      const double* x[kB];
      for (int u = 0; u < kB; ++u) x[u] = reinterpret_cast<const double*>(rows[i0 + std::min(u, ni - 1)] + k0);
      for (int64_t j = i0; j < m; ++j) {
        const double* y = reinterpret_cast<const double*>(rows[j] + k0);
        double re[kB] = {}, im[kB] = {};
        for (int64_t k = 0; k < kn; ++k) {
          const double yr = y[2 * k], yi = y[2 * k + 1];
          for (int u = 0; u < kB; ++u) {
            const double xr = x[u][2 * k], xi = x[u][2 * k + 1];
            re[u] += xr * yr + xi * yi;
            im[u] += xi * yr - xr * yi;
          }
        }
        double* s = &acc[(size_t)(j - i0) * kB * 2];
        for (int u = 0; u < kB; ++u) {
          s[2 * u] += re[u];
          s[2 * u + 1] += im[u];
        }
      }
    }
    for (int64_t j = i0; j < m; ++j)
      for (int u = 0; u < ni && i0 + u <= j; ++u) {
        const double* s = &acc[((size_t)(j - i0) * kB + u) * 2];
        G[(size_t)(i0 + u) * m + j] = cdouble(s[0], s[1]);
      }
  });
}

// ---------------------------------------------------------------------------
// directions (Sec. II.A)
// ---------------------------------------------------------------------------
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kPiD * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int l = 1; l < n; ++l) {
        double p2 = ((2 * l + 1) * z * p1 - l * p0) / (l + 1);
        p0 = p1;
        p1 = p2;
      }
      double pn = (n == 0) ? 1.0 : p1, pm = p0;
      if (n == 1) { pn = z; pm = 1.0; }
      dp = n * (z * pn - pm) / (z * z - 1.0);
      double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute the derivative at the converged node for the weight
    double p0 = 1.0, p1 = z;
    for (int l = 1; l < n; ++l) {
      double p2 = ((2 * l + 1) * z * p1 - l * p0) / (l + 1);
      p0 = p1;
      p1 = p2;
    }
    double pn = p1, pm = p0;
    if (n == 1) { pn = z; pm = 1.0; }
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[n - 1 - i] = z;   // cos guesses decrease with i: store ascending
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

void direction_grid(int L, int nphi, std::vector<double>& khat, std::vector<double>& w) {
  std::vector<double> x, wx;
  gauss_legendre(L + 1, x, wx);
  const int nd = (L + 1) * nphi;
  khat.assign(3 * (size_t)nd, 0.0);
  w.assign(nd, 0.0);
  for (int i = 0; i <= L; ++i) {
    const double st = std::sqrt(std::max(0.0, 1.0 - x[i] * x[i]));
    for (int j = 0; j < nphi; ++j) {
      const double ph = 2.0 * kPiD * j / nphi;
      const int p = i * nphi + j;
      khat[3 * p + 0] = st * std::cos(ph);
      khat[3 * p + 1] = st * std::sin(ph);
      khat[3 * p + 2] = x[i];
      w[p] = wx[i] * 2.0 * kPiD / nphi;
    }
  }
}

// ---------------------------------------------------------------------------
// operator (Eq. 7)
// ---------------------------------------------------------------------------
// h_l^(2)(z), l = 0..L, by upward recurrence from the closed forms
// h_0 = j e^{-jz}/z and h_1 = e^{-jz} (j/z^2 - 1/z); the recurrence is stable
// for the Hankel function as a whole because |h_l| grows with l.  z is
// complex in a lossy medium (Im z < 0, the factor e^{-jz} decays); the
// recurrence never forms j_l and y_l separately, which there are both of
// size e^{|Im z|} and would cancel.
static void hankel2(int L, cdouble z, cdouble* h) {
  const cdouble e = std::exp(cdouble(0.0, -1.0) * z);
  h[0] = cdouble(0.0, 1.0) * e / z;
  if (L >= 1) h[1] = e * (cdouble(0.0, 1.0) / (z * z) - 1.0 / z);
  for (int l = 1; l < L; ++l) h[l + 1] = ((2.0 * l + 1.0) / z) * h[l] - h[l - 1];
}

int multipole_count(double a, double k0, double eps_re, double eps_im, double digits) {
  const double kabs = k0 * std::abs(std::sqrt(cdouble(eps_re, eps_im)));
  const double x = 2.0 * kabs * a * std::sqrt(3.0) / 2.0;
  return (int)std::floor(x + 1.8 * std::cbrt(x) * std::pow(digits, 2.0 / 3.0));
}

static bool is_near(int dx, int dy, int dz, int rule, double kappa) {
  if (dx == 0 && dy == 0 && dz == 0) return true;
  if (rule == 0) return std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) <= 1;
  const double lim = kappa * std::sqrt(3.0) / 2.0;
  return (double)(dx * dx + dy * dy + dz * dz) < lim * lim;
}

void fft_operator(const OperatorSpec& s, const double* khat, std::vector<cdouble>& out) {
  const int n0 = s.n[0], n1 = s.n[1], n2 = s.n[2];
  out.assign((size_t)n0 * n1 * n2, cdouble(0.0, 0.0));
  const int L = s.L;
  const int d2max = (s.K[0] - 1) * (s.K[0] - 1) + (s.K[1] - 1) * (s.K[1] - 1) + (s.K[2] - 1) * (s.K[2] - 1);
  // Hankel values by |d|^2, with the (-j)^l (2l+1) coefficient folded in
  std::vector<cdouble> hc((size_t)(d2max + 1) * (L + 1));
  std::vector<char> seen(d2max + 1, 0);
  const cdouble sq = std::sqrt(cdouble(s.eps_re, s.eps_im));
  const cdouble k = s.k0 * sq;   // wavenumber in the medium
  cdouble pref(1.0, 0.0);
  if (s.prefactor == 1) {
    const cdouble eta = 376.730313668 / sq;
    pref = -k * k * eta / (16.0 * kPiD * kPiD);
  }
  cdouble coef[129];
  {
    cdouble mj(1.0, 0.0);
    for (int l = 0; l <= L; ++l) {
      coef[l] = pref * mj * (2.0 * l + 1.0);
      mj *= cdouble(0.0, -1.0);
    }
  }
  std::vector<cdouble> h(L + 1);
  for (int dz = -(s.K[2] - 1); dz < s.K[2]; ++dz)
    for (int dy = -(s.K[1] - 1); dy < s.K[1]; ++dy)
      for (int dx = -(s.K[0] - 1); dx < s.K[0]; ++dx) {
        if (is_near(dx, dy, dz, s.near_rule, s.kappa)) continue;
        const int d2 = dx * dx + dy * dy + dz * dz;
        if (!seen[d2]) {
          seen[d2] = 1;
          hankel2(L, k * (s.a * std::sqrt((double)d2)), h.data());
          for (int l = 0; l <= L; ++l) hc[(size_t)d2 * (L + 1) + l] = coef[l] * h[l];
        }
        const double inv = 1.0 / std::sqrt((double)d2);
        const double t = (khat[0] * dx + khat[1] * dy + khat[2] * dz) * inv;
        // Legendre P_l(t) by Bonnet's recurrence
        double p0 = 1.0, p1 = t;
        const cdouble* hl = &hc[(size_t)d2 * (L + 1)];
        cdouble acc = hl[0];
        if (L >= 1) acc += hl[1] * p1;
        for (int l = 1; l < L; ++l) {
          const double p2 = ((2 * l + 1) * t * p1 - l * p0) / (l + 1);
          p0 = p1;
          p1 = p2;
          acc += hl[l + 1] * p2;
        }
        const int ix = (dx % n0 + n0) % n0, iy = (dy % n1 + n1) % n1, iz = (dz % n2 + n2) % n2;
        out[((size_t)ix * n1 + iy) * n2 + iz] = acc;
      }
  fft3(out, s.n, -1);
}

// ---------------------------------------------------------------------------
// FFT: iterative radix-2 on contiguous copies of each line
// ---------------------------------------------------------------------------
static void fft_line(cdouble* x, int n, int sign, const cdouble* w /* n/2 roots */) {
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(x[i], x[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    const int half = len / 2, step = n / len;
    for (int i = 0; i < n; i += len)
      for (int k = 0; k < half; ++k) {
        cdouble wk = w[k * step];
        if (sign > 0) wk = std::conj(wk);
        const cdouble u = x[i + k], v = x[i + k + half] * wk;
        x[i + k] = u + v;
        x[i + k + half] = u - v;
      }
  }
}

void fft3(std::vector<cdouble>& a, const int n[3], int sign) {
  const size_t s[3] = {(size_t)n[1] * n[2], (size_t)n[2], 1};
  for (int ax = 0; ax < 3; ++ax) {
    const int m = n[ax];
    std::vector<cdouble> w(m / 2 + 1), line(m);
    for (int k = 0; k < m / 2; ++k) w[k] = std::polar(1.0, -2.0 * kPiD * k / m);
    const int o1 = (ax + 1) % 3, o2 = (ax + 2) % 3;
    for (int i = 0; i < n[o1]; ++i)
      for (int j = 0; j < n[o2]; ++j) {
        cdouble* base = a.data() + i * s[o1] + j * s[o2];
        for (int k = 0; k < m; ++k) line[k] = base[k * s[ax]];
        fft_line(line.data(), m, sign, w.data());
        for (int k = 0; k < m; ++k) base[k * s[ax]] = line[k];
      }
  }
}

// ---------------------------------------------------------------------------
// Hermitian Jacobi eigen-solver
// ---------------------------------------------------------------------------
void hermitian_eig(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V) {
  V.assign((size_t)n * n, cdouble(0.0, 0.0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (auto& z : A) fro += std::norm(z);
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(A[(size_t)p * n + q]);
    if (off <= 1e-32 * fro || off == 0.0) break;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cdouble apq = A[(size_t)p * n + q];
        const double b = std::abs(apq);
        if (b == 0.0) continue;
        const double app = A[(size_t)p * n + p].real(), aqq = A[(size_t)q * n + q].real();
        if (b < 1e-300 || b <= 1e-18 * std::sqrt(std::fabs(app * aqq))) {
          A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
          continue;
        }
        const cdouble ph = apq / b;                  // e^{i phi}
        const double tau = (aqq - app) / (2.0 * b);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        const cdouble sph = s * std::conj(ph);       // s e^{-i phi}
        const cdouble cph = c * std::conj(ph);       // c e^{-i phi}
        const double sr = sph.real(), si = sph.imag(), cr = cph.real(), ci = cph.imag();
        // columns: A <- A V with V = [[c, s], [-s e^{-i phi}, c e^{-i phi}]]
        // (complex products written out: see cdot_conj)
        double* a = reinterpret_cast<double*>(A.data());
        double* v = reinterpret_cast<double*>(V.data());
        for (int k = 0; k < n; ++k) {
          double* x = a + 2 * ((size_t)k * n + p);
          double* y = a + 2 * ((size_t)k * n + q);
          const double xr = x[0], xi = x[1], yr = y[0], yi = y[1];
          x[0] = c * xr - (sr * yr - si * yi);
          x[1] = c * xi - (sr * yi + si * yr);
          y[0] = s * xr + (cr * yr - ci * yi);
          y[1] = s * xi + (cr * yi + ci * yr);
          double* u = v + 2 * ((size_t)k * n + p);
          double* w = v + 2 * ((size_t)k * n + q);
          const double ur = u[0], ui = u[1], wr = w[0], wi = w[1];
          u[0] = c * ur - (sr * wr - si * wi);
          u[1] = c * ui - (sr * wi + si * wr);
          w[0] = s * ur + (cr * wr - ci * wi);
          w[1] = s * ui + (cr * wi + ci * wr);
        }
        // rows: A <- V^H A (conjugated coefficients)
        for (int k = 0; k < n; ++k) {
          double* x = a + 2 * ((size_t)p * n + k);
          double* y = a + 2 * ((size_t)q * n + k);
          const double xr = x[0], xi = x[1], yr = y[0], yi = y[1];
          x[0] = c * xr - (sr * yr + si * yi);
          x[1] = c * xi - (sr * yi - si * yr);
          y[0] = s * xr + (cr * yr + ci * yi);
          y[1] = s * xi + (cr * yi - ci * yr);
        }
        A[(size_t)p * n + q] = A[(size_t)q * n + p] = 0.0;
      }
  }
  std::vector<int> idx(n);
  for (int i = 0; i < n; ++i) idx[i] = i;
  std::stable_sort(idx.begin(), idx.end(), [&](int i, int j) {
    return A[(size_t)i * n + i].real() > A[(size_t)j * n + j].real();
  });
  lam.assign(n, 0.0);
  std::vector<cdouble> Vs((size_t)n * n);
  for (int c = 0; c < n; ++c) {
    lam[c] = A[(size_t)idx[c] * n + idx[c]].real();
    for (int k = 0; k < n; ++k) Vs[(size_t)k * n + c] = V[(size_t)k * n + idx[c]];
  }
  V.swap(Vs);
}

int truncation_rank(const std::vector<double>& lam, double delta, int rule) {
  const int n = (int)lam.size();
  if (n == 0) return 0;
  if (rule == 1) {
    const double s0 = std::sqrt(std::max(lam[0], 0.0));
    for (int j = 0; j < n; ++j)
      if (std::sqrt(std::max(lam[j], 0.0)) < delta * s0) return std::max(j, 1);
    return n;
  }
  // tail[r] = sum_{j >= r} lam_j; smallest r with sqrt(tail) <= delta
  double tail = 0.0;
  int r = n;
  for (int j = n - 1; j >= 0; --j) {
    tail += std::max(lam[j], 0.0);
    if (std::sqrt(tail) <= delta) r = j; else break;
  }
  return std::max(r, 1);
}

// ---------------------------------------------------------------------------
// HOSVD (Alg. 1) for a 3D tensor [n0][n1][n2]
// ---------------------------------------------------------------------------
void hosvd3(const std::vector<cdouble>& T, const int n[3], double gamma, int rule, Tucker3& out) {
  const int n0 = n[0], n1 = n[1], n2 = n[2];
  double norm2 = 0.0;
  for (auto& z : T) norm2 += std::norm(z);
  const double delta = (rule == 0) ? gamma * std::sqrt(norm2) / std::sqrt(3.0) : gamma / std::sqrt(3.0);
  for (int mode = 0; mode < 3; ++mode) {
    const int m = n[mode];
    // Gram matrix of the mode-`mode` unfolding, upper triangle, then mirrored
    std::vector<cdouble> G((size_t)m * m, cdouble(0.0, 0.0));
    if (mode == 0) {
      const size_t len = (size_t)n1 * n2;
      for (int i = 0; i < n0; ++i)
        for (int j = i; j < n0; ++j) G[(size_t)i * m + j] = cdot_conj(&T[i * len], &T[j * len], len);
    } else if (mode == 1) {
      for (int x = 0; x < n0; ++x) {
        const cdouble* S = &T[(size_t)x * n1 * n2];
        for (int i = 0; i < n1; ++i)
          for (int j = i; j < n1; ++j) G[(size_t)i * m + j] += cdot_conj(&S[(size_t)i * n2], &S[(size_t)j * n2], n2);
      }
    } else {
      for (size_t row = 0; row < (size_t)n0 * n1; ++row) {
        const cdouble* v = &T[row * n2];
        for (int i = 0; i < n2; ++i) caxpy_conj(v[i], v + i, &G[(size_t)i * m + i], n2 - i);
      }
    }
    for (int i = 0; i < m; ++i)
      for (int j = i + 1; j < m; ++j) G[(size_t)j * m + i] = std::conj(G[(size_t)i * m + j]);
    std::vector<double> lam;
    std::vector<cdouble> V;
    hermitian_eig_auto(m, G, lam, V);
    const int r = truncation_rank(lam, delta, rule);
    out.r[mode] = r;
    out.U[mode].assign((size_t)m * r, cdouble(0.0, 0.0));
    for (int i = 0; i < m; ++i)
      for (int c = 0; c < r; ++c) out.U[mode][(size_t)i * r + c] = V[(size_t)i * m + c];
  }
  const int r0 = out.r[0], r1 = out.r[1], r2 = out.r[2];
  // Y1[a][y][z] = sum_x conj(U0[x][a]) T[x][y][z]
  std::vector<cdouble> Y1((size_t)r0 * n1 * n2, cdouble(0.0, 0.0));
  const size_t len = (size_t)n1 * n2;
  for (int x = 0; x < n0; ++x)
    for (int a = 0; a < r0; ++a) caxpy(std::conj(out.U[0][(size_t)x * r0 + a]), &T[x * len], &Y1[a * len], len);
  // Y2[a][b][z] = sum_y conj(U1[y][b]) Y1[a][y][z]
  std::vector<cdouble> Y2((size_t)r0 * r1 * n2, cdouble(0.0, 0.0));
  for (int a = 0; a < r0; ++a)
    for (int y = 0; y < n1; ++y)
      for (int b = 0; b < r1; ++b)
        caxpy(std::conj(out.U[1][(size_t)y * r1 + b]), &Y1[((size_t)a * n1 + y) * n2], &Y2[((size_t)a * r1 + b) * n2],
              n2);
  // C[a][b][c] = sum_z conj(U2[z][c]) Y2[a][b][z], with U2 transposed once
  // so that the sum runs over contiguous memory
  std::vector<cdouble> U2h((size_t)r2 * n2);
  for (int z = 0; z < n2; ++z)
    for (int c = 0; c < r2; ++c) U2h[(size_t)c * n2 + z] = std::conj(out.U[2][(size_t)z * r2 + c]);
  out.core.assign((size_t)r0 * r1 * r2, cdouble(0.0, 0.0));
  for (size_t ab = 0; ab < (size_t)r0 * r1; ++ab)
    for (int c = 0; c < r2; ++c) out.core[ab * r2 + c] = cdot(&U2h[(size_t)c * n2], &Y2[ab * n2], n2);
}

}  // namespace fmm
