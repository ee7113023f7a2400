// FP64 host set-up of the translation operators: directions, operator
// samples (Eq. 7), circulant embedding and FFT (Sec. II.B), and the tensor
// decompositions used to compress them (Algs. 1-3).  Independent of the CUDA
// kernels; runs on the host cores.
#pragma once

#include <complex>
#include <cstdint>
#include <functional>
#include <vector>

namespace fmm {

using cdouble = std::complex<double>;

// Run fn(i) for i in [0, n) on the host cores.
void parallel_for(int n, const std::function<void(int)>& fn);

// Complex inner loops of the set-up in explicit real arithmetic.  The
// std::complex operators send every product through the C99 special-value
// handling (a library call per multiply); these compute the textbook
// formulas, which give the same values for finite operands.
// sum_k a[k] conj(b[k])
inline cdouble cdot_conj(const cdouble* a, const cdouble* b, size_t n) {
  const double* x = reinterpret_cast<const double*>(a);
  const double* y = reinterpret_cast<const double*>(b);
  double r0 = 0.0, i0 = 0.0, r1 = 0.0, i1 = 0.0;
  size_t k = 0;
  for (; k + 2 <= n; k += 2) {
    const double* p = x + 2 * k;
    const double* q = y + 2 * k;
    r0 += p[0] * q[0] + p[1] * q[1];
    i0 += p[1] * q[0] - p[0] * q[1];
    r1 += p[2] * q[2] + p[3] * q[3];
    i1 += p[3] * q[2] - p[2] * q[3];
  }
  if (k < n) {
    const double* p = x + 2 * k;
    const double* q = y + 2 * k;
    r0 += p[0] * q[0] + p[1] * q[1];
    i0 += p[1] * q[0] - p[0] * q[1];
  }
  return cdouble(r0 + r1, i0 + i1);
}

// sum_k a[k] b[k]
inline cdouble cdot(const cdouble* a, const cdouble* b, size_t n) {
  const double* x = reinterpret_cast<const double*>(a);
  const double* y = reinterpret_cast<const double*>(b);
  double r0 = 0.0, i0 = 0.0, r1 = 0.0, i1 = 0.0;
  size_t k = 0;
  for (; k + 2 <= n; k += 2) {
    const double* p = x + 2 * k;
    const double* q = y + 2 * k;
    r0 += p[0] * q[0] - p[1] * q[1];
    i0 += p[0] * q[1] + p[1] * q[0];
    r1 += p[2] * q[2] - p[3] * q[3];
    i1 += p[2] * q[3] + p[3] * q[2];
  }
  if (k < n) {
    const double* p = x + 2 * k;
    const double* q = y + 2 * k;
    r0 += p[0] * q[0] - p[1] * q[1];
    i0 += p[0] * q[1] + p[1] * q[0];
  }
  return cdouble(r0 + r1, i0 + i1);
}

// y[k] += u x[k]
inline void caxpy(cdouble u, const cdouble* x, cdouble* y, size_t n) {
  const double ur = u.real(), ui = u.imag();
  const double* X = reinterpret_cast<const double*>(x);
  double* Y = reinterpret_cast<double*>(y);
  for (size_t k = 0; k < n; ++k) {
    const double xr = X[2 * k], xi = X[2 * k + 1];
    Y[2 * k] += ur * xr - ui * xi;
    Y[2 * k + 1] += ur * xi + ui * xr;
  }
}

// y[k] += u conj(x[k])
inline void caxpy_conj(cdouble u, const cdouble* x, cdouble* y, size_t n) {
  const double ur = u.real(), ui = u.imag();
  const double* X = reinterpret_cast<const double*>(x);
  double* Y = reinterpret_cast<double*>(y);
  for (size_t k = 0; k < n; ++k) {
    const double xr = X[2 * k], xi = X[2 * k + 1];
    Y[2 * k] += ur * xr + ui * xi;
    Y[2 * k + 1] += ui * xr - ur * xi;
  }
}

// Upper triangle (j >= i) of the Gram matrix G[i][j] = sum_k x_i[k] conj(x_j[k])
// of m rows of length N (row i at rows[i]); G is m x m row-major, entries
// below the diagonal are left as they are.  Blocks of eight rows meet every
// later row over chunks of the sum, so a block stays in cache while the other
// rows stream past it; the blocks run on the host cores.
void gram_upper(const cdouble* const* rows, int64_t m, int64_t N, cdouble* G);

// Gauss-Legendre nodes (ascending) and weights on [-1, 1], by Newton's method
// on P_n from the asymptotic initial guesses.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w);

// Directions k_p (3 per direction) and weights, theta-major (Sec. II.A).
void direction_grid(int L, int nphi, std::vector<double>& khat, std::vector<double>& w);

struct OperatorSpec {
  int K[3];
  int n[3];
  int L;
  double a, k0;        // k0: free-space wavenumber
  double eps_re, eps_im;  // relative permittivity of the medium (Sec. III.A.5);
                          // k = k0 sqrt(eps_r), eta = eta0 / sqrt(eps_r)
  int near_rule;      // 0 Chebyshev shell max|d_i| <= 1, 1 a|d| < kappa a sqrt(3)/2
  double kappa;
  int prefactor;      // 0 unit, 1 -k^2 eta / (16 pi^2)
};

// Multipole count of the excess-bandwidth rule (Sec. II.A):
// L = floor(2|k|R + 1.8 digits^(2/3) (2|k|R)^(1/3)), R = a sqrt(3)/2 the radius
// of the sphere around a box, |k| = k0 |sqrt(eps_r)|.
int multipole_count(double a, double k0, double eps_re, double eps_im, double digits);

// T~_p = FFT3(embed(T_p)) for direction khat, layout [x][y][z] (z fastest).
void fft_operator(const OperatorSpec& s, const double* khat, std::vector<cdouble>& out);

// In-place unnormalised DFT (sign -1 forward, +1 inverse) of a 3D array
// [n0][n1][n2] (last index fastest), all powers of two.
void fft3(std::vector<cdouble>& a, const int n[3], int sign);

// Eigen-decomposition of a Hermitian n x n matrix (row-major, overwritten) by
// cyclic Jacobi rotations.  Eigenvalues descending in `lam`, eigenvectors as
// the columns of V (row-major n x n).
void hermitian_eig(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V);

// Rank kept at per-step budget delta (rule 0: discarded energy; rule 1:
// first normalised singular value below delta).  lam = squared singular values.
int truncation_rank(const std::vector<double>& lam, double delta, int rule);

struct Tucker3 {
  int r[3];
  std::vector<cdouble> core;   // r1 x r2 x r3
  std::vector<cdouble> U[3];   // n_i x r_i
};

// HOSVD (Alg. 1) of a 3D tensor [n0][n1][n2] at tolerance gamma.
void hosvd3(const std::vector<cdouble>& T, const int n[3], double gamma, int rule, Tucker3& out);

}  // namespace fmm
