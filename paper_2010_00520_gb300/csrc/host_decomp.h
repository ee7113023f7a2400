// FP64 host decompositions of the FFT'ed operators beyond the per-direction
// HOSVD of host_setup.h: TT-SVD of one direction (Alg. 3, 3D format) and the
// 4D-format decompositions of T_4D[x][y][z][p] (Tucker: Alg. 1, H-Tucker:
// Alg. 2, TT: Alg. 3), plus the linear algebra they share.
#pragma once

#include <cstdint>
#include <vector>

#include "host_setup.h"

namespace fmm {

// Eigen-decomposition of a Hermitian n x n matrix (row-major, overwritten):
// eigenvalues descending in `lam`, eigenvectors as the columns of V (row-major
// n x n).  Householder reduction to a real symmetric tridiagonal matrix,
// implicit-shift QL iterations on it, back-transformation.
void hermitian_eig_tridiag(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V);

// Cyclic Jacobi (hermitian_eig) for small n, the tridiagonal route above it.
void hermitian_eig_auto(int n, std::vector<cdouble>& A, std::vector<double>& lam, std::vector<cdouble>& V);

// Per-step truncation budget: the absolute Frobenius budget
// gamma ||T|| / sqrt(parts) for the discarded-energy rule (rule 0), the
// relative threshold gamma / sqrt(parts) for the singular-value rule (rule 1).
double step_budget(double normT, double gamma, double parts, int rule);

// Truncated left singular basis of A (m x N, row-major): U (m x r, orthonormal
// columns) and Q = U^H A (r x N), r from truncation_rank at `delta`.  The
// eigen-decomposition runs on the smaller of A A^H and A^H A.  Returns r.
int truncated_left(const cdouble* A, int64_t m, int64_t N, double delta, int rule,
                   std::vector<cdouble>& U, std::vector<cdouble>& Q);

// TT-SVD (Alg. 3) of one direction T[x][y][z]:
//   T~[x][y][z] = sum_{a,b} U1[x][a] C1[a][y][b] U3[z][b]
struct TT3 {
  int r1 = 0, r2 = 0;
  std::vector<cdouble> U1;   // n1 x r1
  std::vector<cdouble> C1;   // r1 x n2 x r2
  std::vector<cdouble> U3;   // n3 x r2
};
void ttsvd3(const std::vector<cdouble>& T, const int n[3], double gamma, int rule, TT3& out);

// Tucker decomposition of T_4D given by its direction slices Tp[p] (n1 n2 n3,
// [x][y][z]), every mode truncated at the per-step budget `delta`:
//   T_4D = core x_1 U1 x_2 U2 x_3 U3 x_4 U4, core [a][b][c][d] (d fastest)
struct Tucker4 {
  int r[4] = {0, 0, 0, 0};
  std::vector<cdouble> core;
  std::vector<cdouble> U[4];  // n_i x r_i, U4: n_dir x r4
};
void hosvd4(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double delta, int rule, Tucker4& out);

// H-Tucker (Alg. 2), balanced tree {1,2},{3,4}:
//   T_4D[x][y][z][p] = sum U1[x][a] U2[y][b] U3[z][c] U4[p][d]
//                        C12[ab][s] B[s][t] C34[cd][t]
struct HTucker4 {
  int r[6] = {0, 0, 0, 0, 0, 0};   // r1 r2 r3 r4 r12 r34
  std::vector<cdouble> U[4];
  std::vector<cdouble> C12;        // (r1 r2) x r12
  std::vector<cdouble> C34;        // (r3 r4) x r34
  std::vector<cdouble> B;          // r12 x r34
};
void htucker4(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double gamma, int rule, HTucker4& out);

// TT of T_4D (Eq. 14):
//   T_4D[x][y][z][p] = sum U1[x][a] C1[a][y][b] C2[b][z][c] U3[p][c]
struct TT4 {
  int r[3] = {0, 0, 0};
  std::vector<cdouble> U1;   // n1 x r1
  std::vector<cdouble> C1;   // r1 x n2 x r2
  std::vector<cdouble> C2;   // r2 x n3 x r3
  std::vector<cdouble> U3;   // n_dir x r3
};
// TT-SVD of the Tucker core of T_4D (HOSVD first, then Alg. 3 on the core,
// factors absorbed into the cores); budget gamma ||T|| / sqrt(7) per step
// (4 Tucker modes + 3 TT steps), so the total error stays within gamma ||T||.
void tt4_via_tucker(const std::vector<std::vector<cdouble>>& Tp, const int n[3], double gamma, int rule, TT4& out);

}  // namespace fmm
