// Host-side setup tables (Sec. 4.1: Legendre recursion, Gauss-Legendre quadrature, the
// transforms F and B, the matrices D, R, L, RL, LR; Sec. 4.2: the central-flux derivative;
// Sec. 6: the LDG Laplacian with alternating fluxes and jump penalty tau).
#include "dg_tables.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>

namespace dgk {
namespace {

// p_0..p_m at x by (k+1) p_{k+1} = (2k+1) x p_k - k p_{k-1} (Eq. recursion).
void legendre_values(int m, double x, double* p) {
  p[0] = 1.0;
  if (m >= 1) p[1] = x;
  for (int k = 1; k < m; ++k) p[k + 1] = ((2.0 * k + 1.0) * x * p[k] - k * p[k - 1]) / (k + 1.0);
}

// Roots of p_n by Newton's method, p_n' from (x^2 - 1) p_n' = n (x p_n - p_{n-1}).
void gauss_legendre(int n, double* x, double* w) {
  double p[kMaxN + 1];
  for (int j = 0; j < n; ++j) {
    double xj = (n == 1) ? 0.0 : std::cos(M_PI * (j + 0.75) / (n + 0.5));
    for (int it = 0; it < 100 && n > 1; ++it) {
      legendre_values(n, xj, p);
      const double dp = n * (xj * p[n] - p[n - 1]) / (xj * xj - 1.0);
      const double dx = p[n] / dp;
      xj -= dx;
      if (std::fabs(dx) < 1e-17) break;
    }
    legendre_values(n, xj, p);
    const double dp = (n == 1) ? 1.0 : n * (xj * p[n] - p[n - 1]) / (xj * xj - 1.0);
    x[n - 1 - j] = xj;  // the starting guesses decrease with j: store ascending
    w[n - 1 - j] = (n == 1) ? 2.0 : 2.0 / ((1.0 - xj * xj) * dp * dp);
  }
}

using Mat = double[kMaxN][kMaxN];

void matmul(int n, const Mat a, const Mat b, Mat c) {
  Mat t;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += a[i][k] * b[k][j];
      t[i][j] = s;
    }
  std::memcpy(c, t, sizeof(Mat));
}

}  // namespace

int build_ref_tables(int n, double tau, RefTables* t) {
  if (n < 1 || n > kMaxN || !(tau >= 0.0) || t == nullptr) return 1;
  std::memset(t, 0, sizeof(*t));
  t->n = n;
  gauss_legendre(n, t->x, t->w);

  Mat B{}, F{}, D{}, BT{}, Dm{}, G0{};
  double p[kMaxN + 1];
  for (int j = 0; j < n; ++j) {
    legendre_values(n - 1, t->x[j], p);
    for (int k = 0; k < n; ++k) {
      B[j][k] = p[k];                                   // B_{jk} = p_k(x_j)
      F[k][j] = 0.5 * (2.0 * k + 1.0) * t->w[j] * p[k];  // F^{kj} = (2k+1)/2 w_j p_k(x_j)
      BT[j][k] = p[k] * (2.0 * k + 1.0);                // B T^
    }
  }
  double pR[kMaxN], pL[kMaxN];
  for (int k = 0; k < n; ++k) {
    pR[k] = 1.0;
    pL[k] = (k % 2) ? -1.0 : 1.0;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) D[i][j] = (i <= j - 1) ? 1.0 - (((i + j) % 2) ? -1.0 : 1.0) : 0.0;

  // Central derivative: own block B T^ 1/2 (D - D^T) F, face lifts and traces.
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Dm[i][j] = 0.5 * (D[i][j] - D[j][i]);
  Mat tmp;
  matmul(n, BT, Dm, tmp);
  matmul(n, tmp, F, t->C0);
  double liftR[kMaxN], liftL[kMaxN];  // B T^ p(+1), B T^ p(-1)
  for (int i = 0; i < n; ++i) {
    liftR[i] = liftL[i] = 0.0;
    for (int k = 0; k < n; ++k) {
      liftR[i] += BT[i][k] * pR[k];
      liftL[i] += BT[i][k] * pL[k];
    }
    t->muR[i] = 0.5 * liftR[i];
    t->muL[i] = 0.5 * liftL[i];
  }
  for (int j = 0; j < n; ++j) {
    t->lL[j] = t->lR[j] = 0.0;
    for (int k = 0; k < n; ++k) {
      t->lL[j] += F[k][j] * pL[k];
      t->lR[j] += F[k][j] * pR[k];
    }
  }

  // LDG: forward derivative D+ (flux from the right cell), per unit h:
  //   own block G0 = B T^ (-L - D^T) F, right-neighbour block Gp = liftR lL^T.
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Dm[i][j] = -pL[i] * pL[j] - D[j][i];
  matmul(n, BT, Dm, tmp);
  matmul(n, tmp, F, G0);
  double wh[kMaxN];
  for (int j = 0; j < n; ++j) wh[j] = 0.5 * t->w[j];
  // A1 = D+^T W D+ + tau sum_f j_f j_f^T  (per unit h); blocks:
  //   (c,c)   G0^T W G0 + gamma lL lL^T + tau (lL lL^T + lR lR^T),  gamma = liftR^T W liftR
  //   (c,c+1) beta lL^T with beta = G0^T W liftR - tau lR;  (c,c-1) = its transpose.
  double gamma = 0.0;
  for (int j = 0; j < n; ++j) gamma += liftR[j] * wh[j] * liftR[j];
  double A1[kMaxN][kMaxN], beta[kMaxN];
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += G0[k][i] * wh[k] * G0[k][j];
      A1[i][j] = s + gamma * t->lL[i] * t->lL[j] + tau * (t->lL[i] * t->lL[j] + t->lR[i] * t->lR[j]);
    }
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += G0[k][i] * wh[k] * liftR[k];
    beta[i] = s - tau * t->lR[i];
  }
  std::memcpy(t->A1cc, A1, sizeof(A1));
  std::memcpy(t->betaA, beta, sizeof(beta));

  // Dirichlet first cell: G0' = B T^ (-D^T) F (the left-face term -L dropped: u^ = 0 there).
  Mat G0d{};
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Dm[i][j] = -D[j][i];
  matmul(n, BT, Dm, tmp);
  matmul(n, tmp, F, G0d);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += G0d[k][i] * wh[k] * G0d[k][j];
      t->A1first[i][j] = s + kDirichletPenalty * t->lL[i] * t->lL[j];
    }
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += G0d[k][i] * wh[k] * liftR[k];
    t->betaFirst[i] = s;
  }
  return 0;
}

int hermitian_eig(int m, const long double* Hre, const long double* Him, double* lam, double* Vre, double* Vim) {
  using R = long double;
  using cd = std::complex<R>;
  cd H[kMaxN][kMaxN], V[kMaxN][kMaxN];
  R fro = 0.0L;
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      H[i][j] = cd(Hre[i * m + j], Him[i * m + j]);
      V[i][j] = cd(i == j ? 1.0L : 0.0L, 0.0L);
      fro += std::norm(H[i][j]);
    }
  fro = std::sqrt(fro);
  bool done = m < 2 || fro == 0.0L;
  for (int sweep = 0; sweep < 60 && !done; ++sweep) {
    R off = 0.0L;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        if (i != j) off += std::norm(H[i][j]);
    if (std::sqrt(off) <= 1e-18L * fro) {
      done = true;
      break;
    }
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        const R beta = std::abs(H[p][q]);
        if (beta == 0.0L) continue;
        // U = D R: D_qq = e^{-i phi} makes the (p, q) entry real (|h_pq|), R the plane rotation
        // with R_pp = R_qq = c, R_pq = s, R_qp = -s that zeroes it.
        const cd e = std::conj(H[p][q]) / beta;  // e^{-i phi}
        const R alpha = H[p][p].real(), gamma = H[q][q].real();
        const R tau = (gamma - alpha) / (2.0L * beta);
        const R t = (tau >= 0.0L ? 1.0L : -1.0L) / (std::fabs(tau) + std::sqrt(1.0L + tau * tau));
        const R c = 1.0L / std::sqrt(1.0L + t * t), s = t * c;
        const cd Upp = c, Upq = s, Uqp = -s * e, Uqq = c * e;
        // H <- U^* H U (columns p, q, then rows p, q), V <- V U
        for (int i = 0; i < m; ++i) {
          const cd hp = H[i][p], hq = H[i][q];
          H[i][p] = hp * Upp + hq * Uqp;
          H[i][q] = hp * Upq + hq * Uqq;
          const cd vp = V[i][p], vq = V[i][q];
          V[i][p] = vp * Upp + vq * Uqp;
          V[i][q] = vp * Upq + vq * Uqq;
        }
        for (int j = 0; j < m; ++j) {
          const cd hp = H[p][j], hq = H[q][j];
          H[p][j] = std::conj(Upp) * hp + std::conj(Uqp) * hq;
          H[q][j] = std::conj(Upq) * hp + std::conj(Uqq) * hq;
        }
        H[p][q] = H[q][p] = 0.0L;
        H[p][p] = H[p][p].real();
        H[q][q] = H[q][q].real();
      }
  }
  if (!done) {
    R off = 0.0L;
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        if (i != j) off += std::norm(H[i][j]);
    if (std::sqrt(off) > 1e-15L * fro) return -1;
  }
  int order[kMaxN];
  for (int i = 0; i < m; ++i) order[i] = i;
  std::sort(order, order + m, [&](int x, int y) { return H[x][x].real() < H[y][y].real(); });
  for (int j = 0; j < m; ++j) {
    lam[j] = double(H[order[j]][order[j]].real());
    for (int i = 0; i < m; ++i) {
      Vre[i * m + j] = double(V[i][order[j]].real());
      Vim[i * m + j] = double(V[i][order[j]].imag());
    }
  }
  return 0;
}

}  // namespace dgk
