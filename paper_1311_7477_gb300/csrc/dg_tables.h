// Host-side setup tables of the dG method (Sec. 4.1-4.2 and the LDG Laplacian of Sec. 6).
//
// All tables are dimensionless (reference cell [-1, 1]); the kernels scale them by the
// cell sizes.  n = P = number of Gauss nodes / Legendre polynomials per dimension (1..5).
#pragma once

namespace dgk {

constexpr int kMaxN = 5;

struct RefTables {
  int n;
  double x[kMaxN], w[kMaxN];        // Gauss-Legendre abscissas and weights on [-1, 1]
  // Central-flux derivative (Eq. discrete_der mapped to X-space, Eq. matrix_xspace):
  //   h * (f_x)_c = C0 f_c + muR (lL . f_{c+1}) - muL (lR . f_{c-1})
  double C0[kMaxN][kMaxN];          // B T^ 1/2 (D - D^T) F,   T^ = diag(2k+1)
  double muR[kMaxN], muL[kMaxN];    // 1/2 B T^ p(+1), 1/2 B T^ p(-1)
  double lL[kMaxN], lR[kMaxN];      // F^T p(-1), F^T p(+1): face values from nodal values
  // LDG stiffness A1 = D+^T W D+ + tau sum_f j_f j_f^T (1D, per unit h; Sec. 6):
  //   h * (A1 u)_c = A1cc u_c + betaA (lL . u_{c+1}) + lL (betaA . u_{c-1})
  double A1cc[kMaxN][kMaxN];
  double betaA[kMaxN];
  // Homogeneous Dirichlet boundaries: the first cell's diagonal block of A1 (per unit h) when
  // the forward derivative's flux on the left boundary face is the boundary value u^ = 0
  // (own block G0' = B T^ (-D^T) F) and the trace is penalised there:
  //   A1first = G0'^T W G0' + kDirichletPenalty lL lL^T   (no right-neighbour term from the left)
  double A1first[kMaxN][kMaxN];
  // ... and its coupling to the second cell: h (A1 u)_0 = A1first u_0 + betaFirst (lL . u_1),
  // h (A1 u)_1 = ... + lL (betaFirst . u_0), betaFirst = G0'^T W B T^ p(+1)
  double betaFirst[kMaxN];
};

constexpr double kDirichletPenalty = 1.0;  // (penalty / h) u(a)^2 on the left boundary face

// Fills t for 1 <= n <= kMaxN and penalty tau >= 0.  Returns 0 on success.
int build_ref_tables(int n, double tau, RefTables* t);

// Eigen-decomposition of a Hermitian m x m matrix (m <= kMaxN) given row-major by its real and
// imaginary parts: H = V diag(lam) V^*, V unitary (column j = eigenvector j), lam ascending.
// Cyclic Jacobi rotations, each of which zeroes one off-diagonal pair (a phase that makes the
// pair real, then a real plane rotation), in long double: the small eigenvalues of the
// operators' symbols (about 1 against 1e7 and more) then come out accurate to float64
// precision.  Returns 0, or -1 when the off-diagonal part is not below 1e-15 of the matrix's
// Frobenius norm after 60 sweeps.
int hermitian_eig(int m, const long double* Hre, const long double* Him, double* lam, double* Vre, double* Vim);

}  // namespace dgk
