// The C ABI of libdgk (include/dg.h): handles, argument checks, operator tables, kernel
// launches and the time-stepper orchestration.  No function here aborts or prints; errors
// are returned as DG_ERR_* with a thread-local message.
#include "dg_host.cuh"

namespace dgk {
thread_local char g_err[512] = "";
}  // namespace dgk

namespace {

template <typename T, int N>
void fill_op(Op1D<T, N>& o, const double M[kMaxN][kMaxN], const double* a, const double* r, const double* d,
             const double* s, const double Mf[kMaxN][kMaxN] = nullptr, const double* af = nullptr,
             const double* sf = nullptr) {
  for (int i = 0; i < N; ++i) {
    for (int j = 0; j < N; ++j) o.M[i][j] = T(M[i][j]);
    for (int j = 0; j < N; ++j) o.Mf[i][j] = T(Mf ? Mf[i][j] : M[i][j]);
    o.af[i] = T(af ? af[i] : a[i]);
    o.sf[i] = T(sf ? sf[i] : s[i]);
    o.a[i] = T(a[i]);
    o.r[i] = T(r[i]);
    o.d[i] = T(d[i]);
    o.s[i] = T(s[i]);
  }
}

// Builds the 2D operator tables from the dimensionless per-n tables (Sec. 4.2 / Sec. 6)
// (the LDG operators' Mf: the first cell's own block at a Dirichlet boundary, A1first):
//   d/dx   = C0/hx, lifts muR/hx and -muL/hx on the traces lL . u_{c+1}, lR . u_{c-1};
//   -Delta = W^-1 A (x-part: w^-1 A1cc / hx^2, w^-1 betaA / hx^2 on lL . u_{c+1},
//            w^-1 lL / hx^2 on betaA . u_{c-1});
//   W^-1/2 A W^-1/2 = the same with w^-1/2 on both sides.
template <typename T, int N>
Ops2D<T, N> make_ops(const RefTables& t, double hx, double hy) {
  Ops2D<T, N> O;
  double wh[kMaxN], rw[kMaxN];
  for (int j = 0; j < N; ++j) {
    wh[j] = 0.5 * t.w[j];
    rw[j] = 1.0 / std::sqrt(wh[j]);
  }
  const double hs[2] = {hx, hy};
  for (int dir = 0; dir < 2; ++dir) {
    const double h = hs[dir], h2 = h * h;
    double M[kMaxN][kMaxN], a[kMaxN], r[kMaxN], d[kMaxN], s[kMaxN], Mf[kMaxN][kMaxN], af[kMaxN], sf[kMaxN];
    // central derivative
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) M[i][j] = t.C0[i][j] / h;
      a[i] = t.muR[i] / h;
      r[i] = t.lL[i];
      d[i] = -t.muL[i] / h;
      s[i] = t.lR[i];
    }
    fill_op<T, N>(dir == 0 ? O.dx : O.dy, M, a, r, d, s);
    // symmetrically scaled LDG stiffness
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) M[i][j] = rw[i] * t.A1cc[i][j] * rw[j] / h2;
      for (int j = 0; j < N; ++j) Mf[i][j] = rw[i] * t.A1first[i][j] * rw[j] / h2;
      a[i] = rw[i] * t.betaA[i] / h2;
      r[i] = rw[i] * t.lL[i];
      d[i] = rw[i] * t.lL[i] / h2;
      s[i] = rw[i] * t.betaA[i];
      af[i] = rw[i] * t.betaFirst[i] / h2;
      sf[i] = rw[i] * t.betaFirst[i];
    }
    fill_op<T, N>(dir == 0 ? O.kx : O.ky, M, a, r, d, s, Mf, af, sf);
    // -Delta_h = W^-1 A
    for (int i = 0; i < N; ++i) {
      for (int j = 0; j < N; ++j) M[i][j] = t.A1cc[i][j] / (wh[i] * h2);
      for (int j = 0; j < N; ++j) Mf[i][j] = t.A1first[i][j] / (wh[i] * h2);
      a[i] = t.betaA[i] / (wh[i] * h2);
      r[i] = t.lL[i];
      d[i] = t.lL[i] / (wh[i] * h2);
      s[i] = t.betaA[i];
      af[i] = t.betaFirst[i] / (wh[i] * h2);
      sf[i] = t.betaFirst[i];
    }
    fill_op<T, N>(dir == 0 ? O.lx : O.ly, M, a, r, d, s, Mf, af, sf);
  }
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double w = (hy * wh[a]) * (hx * wh[b]);
      O.wq[a * N + b] = T(w);
      O.sw[a * N + b] = T(std::sqrt(w));
      O.isw[a * N + b] = T(1.0 / std::sqrt(w));
    }
  return O;
}

}  // namespace

namespace {

void free_ws(Workspace& w) {
  cudaFree(w.r);
  cudaFree(w.p0);
  cudaFree(w.p1);
  cudaFree(w.q);
  cudaFree(w.y);
  cudaFree(w.part);
  cudaFree(w.sync);
  cudaFree(w.status);
  cudaFree(w.inv_part);
  cudaFree(w.inv_out);
  cudaFree(w.rf);
  cudaFree(w.fr);
  cudaFree(w.fe);
  cudaFree(w.fp0);
  cudaFree(w.fp1);
  cudaFree(w.fq);
  cudaFree(w.partf);
  cudaFree(w.pz);
  cudaFree(w.prc);
  cudaFree(w.puc);
  cudaFree(w.pC);
  cudaFree(w.pzf);
  cudaFree(w.prcf);
  cudaFree(w.pucf);
  cudaFree(w.pCf);
  cudaFree(w.pS);
  cudaFree(w.pSf);
  if (w.host_out) cudaFreeHost(w.host_out);
  w = Workspace{};
}

int alloc_ws(Workspace& w, size_t ndof, int grid_cap, bool with_y) {
  w.ndof = ndof;
  w.grid_cap = grid_cap;
  const size_t bytes = ndof * sizeof(double);
  CUDA_TRY(cudaMalloc(&w.r, bytes));
  CUDA_TRY(cudaMalloc(&w.p0, bytes));
  CUDA_TRY(cudaMalloc(&w.p1, bytes));
  CUDA_TRY(cudaMalloc(&w.q, bytes));
  if (with_y) CUDA_TRY(cudaMalloc(&w.y, bytes));
  CUDA_TRY(cudaMalloc(&w.part, 6 * (size_t)grid_cap * sizeof(double)));
  CUDA_TRY(cudaMalloc(&w.sync, sizeof(SyncState)));
  CUDA_TRY(cudaMalloc(&w.status, sizeof(SolveStatus)));
  CUDA_TRY(cudaMemset(w.sync, 0, sizeof(SyncState)));
  CUDA_TRY(cudaMemset(w.status, 0, sizeof(SolveStatus)));
  CUDA_TRY(cudaMalloc(&w.inv_part, 3 * (size_t)kInvBlocks * sizeof(double)));
  CUDA_TRY(cudaMalloc(&w.inv_out, 3 * sizeof(double)));
  CUDA_TRY(cudaMallocHost(&w.host_out, 3 * sizeof(double)));
  return DG_OK;
}

// Preconditioner work arrays for a grid of Nx x Ny cells with n nodes per side: the two-level
// vectors and the spectral preconditioner's spectrum ((Nx/2 + 1) Ny n^2 complex values),
// float64 and, for the mixed modes, float32.
int alloc_ws_precond(Workspace& w, int Nx, int Ny, int n, bool mixed) {
  const size_t ncell = (size_t)Nx * Ny;
  const size_t nspec = (size_t)(Nx / 2 + 1) * Ny * n * n;
  CUDA_TRY(cudaMalloc(&w.pz, w.ndof * sizeof(double)));
  CUDA_TRY(cudaMalloc(&w.prc, ncell * sizeof(double)));
  CUDA_TRY(cudaMalloc(&w.puc, ncell * sizeof(double)));
  CUDA_TRY(cudaMalloc(&w.pC, ncell * sizeof(Cplx<double>)));
  CUDA_TRY(cudaMalloc(&w.pS, nspec * sizeof(Cplx<double>)));
  if (mixed) {
    CUDA_TRY(cudaMalloc(&w.pzf, w.ndof * sizeof(float)));
    CUDA_TRY(cudaMalloc(&w.prcf, ncell * sizeof(float)));
    CUDA_TRY(cudaMalloc(&w.pucf, ncell * sizeof(float)));
    CUDA_TRY(cudaMalloc(&w.pCf, ncell * sizeof(Cplx<float>)));
    CUDA_TRY(cudaMalloc(&w.pSf, nspec * sizeof(Cplx<float>)));
  }
  return DG_OK;
}

int alloc_ws_mixed(Workspace& w) {
  const size_t fb = w.ndof * sizeof(float);
  CUDA_TRY(cudaMalloc(&w.rf, fb));
  CUDA_TRY(cudaMalloc(&w.fr, fb));
  CUDA_TRY(cudaMalloc(&w.fe, fb));
  CUDA_TRY(cudaMalloc(&w.fp0, fb));
  CUDA_TRY(cudaMalloc(&w.fp1, fb));
  CUDA_TRY(cudaMalloc(&w.fq, fb));
  CUDA_TRY(cudaMalloc(&w.partf, 6 * (size_t)w.grid_cap * sizeof(float)));
  return DG_OK;
}

// Gershgorin bound on the largest eigenvalue of the CG operator Ahat = I (x) kx + ky (x) I:
// the largest row sum of |kx| plus that of |ky| (a row of a 1D operator couples the cell's own
// nodes through M and the neighbours' face traces through a r^T and d s^T).
template <int N>
double ahat_row_bound(const Ops2D<double, N>& O) {
  auto rowsum = [](const Op1D<double, N>& o) {
    double sr = 0.0, ss = 0.0, m = 0.0;
    for (int j = 0; j < N; ++j) {
      sr += std::fabs(o.r[j]);
      ss += std::fabs(o.s[j]);
    }
    for (int i = 0; i < N; ++i) {
      double t = std::fabs(o.a[i]) * sr + std::fabs(o.d[i]) * ss;
      for (int j = 0; j < N; ++j) t += std::fabs(o.M[i][j]);
      m = std::max(m, t);
    }
    return m;
  };
  return rowsum(O.kx) + rowsum(O.ky);
}

// Whether a float32 evaluation of the CG operator Ahat is too inexact on the grid's smoothest
// modes for the float32 inner solve of the mixed modes.  Its absolute error is about eps32
// times the row sums of |Ahat|, against the smallest non-zero eigenvalue of -Delta on the
// periodic box, min((2 pi / Lx)^2, (2 pi / Ly)^2); once that ratio exceeds 0.05 (512^2 cells
// with n >= 4, 1024^2 with n >= 3 on [0, 2 pi]^2) the inner solves switch to the double-float
// apply when a refinement sweep stalls (dg_grid_set_compensated_apply overrides the choice).
template <int N>
bool precise_apply_needed(const Ops2D<double, N>& O, double Lx, double Ly, int bc) {
  const double lam_min = bc == DG_BC_PERIODIC
                             ? std::min(std::pow(2.0 * M_PI / Lx, 2), std::pow(2.0 * M_PI / Ly, 2))
                             : std::pow(M_PI / Lx, 2) + std::pow(M_PI / Ly, 2);
  return std::ldexp(ahat_row_bound<N>(O), -24) / lam_min > 0.05;
}

template <int N>
void build_ops(dg_grid* g) {
  new (g->ops.d) Ops2D<double, N>(make_ops<double, N>(g->rt, g->hx, g->hy));
  new (g->ops.f) Ops2D<float, N>(make_ops<float, N>(g->rt, g->hx, g->hy));
  const Ops2D<df, N> x = make_ops<df, N>(g->rt, g->hx, g->hy);
  new (g->ops.x) Ops2D<df, N>(x);
  new (g->ops.k) OpsK<df, N>(OpsK<df, N>{x.kx, x.ky});
  const Ops2D<double, N>& Od = *reinterpret_cast<const Ops2D<double, N>*>(g->ops.d);
  g->precise_auto = precise_apply_needed<N>(Od, g->Lx, g->Ly, g->bc) ? 2 : 0;
  g->precise_apply = g->precise_auto;
  const double f = std::ldexp(ahat_row_bound<N>(Od), -52);
  g->floor2 = f * f;
}

// ---- two-level preconditioner tables ---------------------------------------------------

void free_pc(PcTables& t) {
  cudaFree(t.Bt);
  cudaFree(t.twx);
  cudaFree(t.twy);
  cudaFree(t.ax);
  cudaFree(t.ay);
  cudaFree(t.Btf);
  cudaFree(t.twxf);
  cudaFree(t.twyf);
  cudaFree(t.axf);
  cudaFree(t.ayf);
  cudaFree(t.Vx);
  cudaFree(t.Vy);
  cudaFree(t.lx);
  cudaFree(t.ly);
  cudaFree(t.Vxf);
  cudaFree(t.Vyf);
  cudaFree(t.lxf);
  cudaFree(t.lyf);
  t = PcTables{};
}

int log2_exact(int L) {
  int k = 0;
  while ((1 << k) < L) ++k;
  return (1 << k) == L ? k : -1;
}

// Gauss-Jordan inverse with partial pivoting of an m x m matrix (row-major, in place into inv).
bool invert(int m, std::vector<double> a, std::vector<double>& inv) {
  inv.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; ++i) inv[(size_t)i * m + i] = 1.0;
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(a[(size_t)r * m + c]) > std::fabs(a[(size_t)piv * m + c])) piv = r;
    if (a[(size_t)piv * m + c] == 0.0) return false;
    for (int j = 0; j < m; ++j) {
      std::swap(a[(size_t)c * m + j], a[(size_t)piv * m + j]);
      std::swap(inv[(size_t)c * m + j], inv[(size_t)piv * m + j]);
    }
    const double d = 1.0 / a[(size_t)c * m + c];
    for (int j = 0; j < m; ++j) {
      a[(size_t)c * m + j] *= d;
      inv[(size_t)c * m + j] *= d;
    }
    for (int r = 0; r < m; ++r) {
      if (r == c) continue;
      const double f = a[(size_t)r * m + c];
      if (f == 0.0) continue;
      for (int j = 0; j < m; ++j) {
        a[(size_t)r * m + j] -= f * a[(size_t)c * m + j];
        inv[(size_t)r * m + j] -= f * inv[(size_t)c * m + j];
      }
    }
  }
  return true;
}

template <typename H, typename D>
int upload(D** dst, const std::vector<H>& src) {
  std::vector<D> tmp(src.size());
  for (size_t i = 0; i < src.size(); ++i) tmp[i] = D(src[i]);
  CUDA_TRY(cudaMalloc(dst, tmp.size() * sizeof(D)));
  CUDA_TRY(cudaMemcpy(*dst, tmp.data(), tmp.size() * sizeof(D), cudaMemcpyHostToDevice));
  return DG_OK;
}

int upload_tw(int L, Cplx<double>** d, Cplx<float>** f) {
  std::vector<Cplx<double>> tw(L);
  std::vector<Cplx<float>> twf(L);
  for (int m = 0; m < L; ++m) {
    const double ang = 2.0 * M_PI * double(m) / double(L);
    tw[m] = Cplx<double>{std::cos(ang), -std::sin(ang)};
    twf[m] = Cplx<float>{float(tw[m].re), float(tw[m].im)};
  }
  CUDA_TRY(cudaMalloc(d, L * sizeof(Cplx<double>)));
  CUDA_TRY(cudaMemcpy(*d, tw.data(), L * sizeof(Cplx<double>), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(f, L * sizeof(Cplx<float>)));
  CUDA_TRY(cudaMemcpy(*f, twf.data(), L * sizeof(Cplx<float>), cudaMemcpyHostToDevice));
  return DG_OK;
}

// ---- spectral preconditioner tables -------------------------------------------------------

// The symbol of a scaled 1D CG operator on a periodic line of Nc cells at wave number k,
// K(k) = M + e^{i th} a r^T + e^{-i th} d s^T with th = 2 pi k / Nc (from (Op u)_c = M u_c +
// a (r . u_{c+1}) + d (s . u_{c-1}) and u_c = sum_k u^_k e^{i th c}), and its eigen-decomposition
// K = V diag(lam) V^* (row-major V, column j = eigenvector j, lam ascending).  K is Hermitian
// because the operator is symmetric; its parts are symmetrised before the decomposition.  At
// k = 0 the smallest eigenvalue is the constant mode's, rounding-sized: it is set to exactly 0.
template <int N>
int spectral_symbol(const Op1D<double, N>& o, int Nc, int k, double* lam, double* Vre, double* Vim) {
  // in long double: at small k the terms of the symbol cancel to a smallest eigenvalue ~1e-7
  // of the largest, which float64 would leave with a relative error of ~1e-9
  using R = long double;
  const R pi = 3.141592653589793238462643383279502884L;
  const R th = 2.0L * pi * R(k) / R(Nc);
  const R c = std::cos(th), sn = std::sin(th);
  R Kre[N * N], Kim[N * N];
  for (int b = 0; b < N; ++b)
    for (int j = 0; j < N; ++j) {
      Kre[b * N + j] = R(o.M[b][j]) + c * (R(o.a[b]) * R(o.r[j]) + R(o.d[b]) * R(o.s[j]));
      Kim[b * N + j] = sn * (R(o.a[b]) * R(o.r[j]) - R(o.d[b]) * R(o.s[j]));
    }
  for (int b = 0; b < N; ++b)
    for (int j = b; j < N; ++j) {
      const R re = 0.5L * (Kre[b * N + j] + Kre[j * N + b]);
      const R im = 0.5L * (Kim[b * N + j] - Kim[j * N + b]);
      Kre[b * N + j] = Kre[j * N + b] = re;
      Kim[b * N + j] = im;
      Kim[j * N + b] = -im;
    }
  if (hermitian_eig(N, Kre, Kim, lam, Vre, Vim)) return fail(DG_ERR_ARG, "eigen-decomposition of the symbol did not converge");
  if (k == 0) {
    // the constant mode: zero up to the rounding of the (cancelling) sum of the blocks
    double big = 0.0;
    for (int b = 0; b < N; ++b)
      for (int j = 0; j < N; ++j)
        big = std::max({big, std::fabs(o.M[b][j]), std::fabs(o.a[b] * o.r[j]), std::fabs(o.d[b] * o.s[j])});
    if (std::fabs(lam[0]) > 1e-9 * big) return fail(DG_ERR_ARG, "the symbol at k = 0 has no null mode");
    lam[0] = 0.0;
  }
  return DG_OK;
}

// Vx / lx for kx = 0 .. Nx/2 and Vy / ly for ky = 0 .. Ny - 1 (PrecondArgs), float64 and float32.
template <int N>
int build_spectral(dg_grid* g) {
  const Ops2D<double, N>& O = *reinterpret_cast<const Ops2D<double, N>*>(g->ops.d);
  PcTables& P = g->pc;
  auto line = [&](const Op1D<double, N>& o, int Nc, int kcount, Cplx<double>** V, double** lam, Cplx<float>** Vf,
                  float** lamf) {
    std::vector<Cplx<double>> vh((size_t)kcount * N * N);
    std::vector<Cplx<float>> vf((size_t)kcount * N * N);
    std::vector<double> lh((size_t)kcount * N);
    for (int k = 0; k < kcount; ++k) {
      double l[N], vre[N * N], vim[N * N];
      if (int rc = spectral_symbol<N>(o, Nc, k, l, vre, vim)) return rc;
      for (int i = 0; i < N * N; ++i) {
        vh[(size_t)k * N * N + i] = Cplx<double>{vre[i], vim[i]};
        vf[(size_t)k * N * N + i] = Cplx<float>{float(vre[i]), float(vim[i])};
      }
      for (int i = 0; i < N; ++i) lh[(size_t)k * N + i] = l[i];
    }
    CUDA_TRY(cudaMalloc(V, vh.size() * sizeof(Cplx<double>)));
    CUDA_TRY(cudaMemcpy(*V, vh.data(), vh.size() * sizeof(Cplx<double>), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMalloc(Vf, vf.size() * sizeof(Cplx<float>)));
    CUDA_TRY(cudaMemcpy(*Vf, vf.data(), vf.size() * sizeof(Cplx<float>), cudaMemcpyHostToDevice));
    if (int rc = upload(lam, lh)) return rc;
    return upload(lamf, lh);
  };
  if (int rc = line(O.kx, g->Nx, g->Nx / 2 + 1, &P.Vx, &P.lx, &P.Vxf, &P.lxf)) return rc;
  return line(O.ky, g->Ny, g->Ny, &P.Vy, &P.ly, &P.Vyf, &P.lyf);
}

// The cell block A_cc = W_y (x) A1_cc/hx + A1_cc/hy (x) W_x (node index a*n + b), its inverse
// scaled by sqrt(W) on both sides; the coarse eigenvalues of P^T A P from the 1D cell-average
// stencil [co, cc, co] (cc = 1^T A1_cc 1, co = (1^T betaA)(1^T lL), per unit h):
// lambda(kx, ky) = (hy/hx)(cc + 2 co cos(2 pi kx/Nx)) + (hx/hy)(cc + 2 co cos(2 pi ky/Ny)).
int build_pc(dg_grid* g) {
  const int n = g->n, NN = n * n;
  const RefTables& t = g->rt;
  double wh[kMaxN];
  for (int j = 0; j < n; ++j) wh[j] = 0.5 * t.w[j];
  std::vector<double> Acc((size_t)NN * NN, 0.0);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int a2 = 0; a2 < n; ++a2)
        for (int b2 = 0; b2 < n; ++b2) {
          double v = 0.0;
          if (a == a2) v += g->hy * wh[a] * t.A1cc[b][b2] / g->hx;
          if (b == b2) v += t.A1cc[a][a2] / g->hy * g->hx * wh[b];
          Acc[(size_t)(a * n + b) * NN + (a2 * n + b2)] = v;
        }
  std::vector<double> inv;
  if (!invert(NN, Acc, inv)) return fail(DG_ERR_ARG, "cell block of the LDG operator is singular");
  std::vector<double> sw(NN);
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) sw[a * n + b] = std::sqrt(g->hy * wh[a] * g->hx * wh[b]);
  std::vector<double> Bt((size_t)NN * NN);
  for (int k = 0; k < NN; ++k)
    for (int j = 0; j < NN; ++j) Bt[(size_t)k * NN + j] = sw[k] * inv[(size_t)k * NN + j] * sw[j];
  double cc = 0.0, sb = 0.0, sl = 0.0;
  for (int i = 0; i < n; ++i) {
    for (int j = 0; j < n; ++j) cc += t.A1cc[i][j];
    sb += t.betaA[i];
    sl += t.lL[i];
  }
  const double co = sb * sl;
  std::vector<double> ax(g->Nx), ay(g->Ny);
  for (int k = 0; k < g->Nx; ++k) ax[k] = (g->hy / g->hx) * (cc + 2.0 * co * std::cos(2.0 * M_PI * k / g->Nx));
  for (int k = 0; k < g->Ny; ++k) ay[k] = (g->hx / g->hy) * (cc + 2.0 * co * std::cos(2.0 * M_PI * k / g->Ny));
  PcTables& P = g->pc;
  if (int rc = upload(&P.Bt, Bt)) return rc;
  if (int rc = upload(&P.Btf, Bt)) return rc;
  if (int rc = upload(&P.ax, ax)) return rc;
  if (int rc = upload(&P.axf, ax)) return rc;
  if (int rc = upload(&P.ay, ay)) return rc;
  if (int rc = upload(&P.ayf, ay)) return rc;
  if (int rc = upload_tw(g->Nx, &P.twx, &P.twxf)) return rc;
  if (int rc = upload_tw(g->Ny, &P.twy, &P.twyf)) return rc;
  P.log2x = log2_exact(g->Nx);
  P.log2y = log2_exact(g->Ny);
  // the spectral tables: their failure (reported by dg_grid_set_precond) leaves the grid usable
  if (g->bc == DG_BC_PERIODIC) {
    P.spectral_rc = dispatch_n(n, [&](auto nc) { return build_spectral<decltype(nc)::value>(g); });
    if (P.spectral_rc == DG_ERR_CUDA || P.spectral_rc == DG_ERR_NOMEM) return P.spectral_rc;
  }
  return DG_OK;
}

int upload_ops(dg_grid* g) {
  CUDA_TRY(cudaMalloc(&g->d_opsd, sizeof(g->ops.d)));
  CUDA_TRY(cudaMemcpy(g->d_opsd, g->ops.d, sizeof(g->ops.d), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(&g->d_opsf, sizeof(g->ops.f)));
  CUDA_TRY(cudaMemcpy(g->d_opsf, g->ops.f, sizeof(g->ops.f), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(&g->d_opsx, sizeof(g->ops.x)));
  CUDA_TRY(cudaMemcpy(g->d_opsx, g->ops.x, sizeof(g->ops.x), cudaMemcpyHostToDevice));
  CUDA_TRY(cudaMalloc(&g->d_opsk, sizeof(g->ops.k)));
  CUDA_TRY(cudaMemcpy(g->d_opsk, g->ops.k, sizeof(g->ops.k), cudaMemcpyHostToDevice));
  return DG_OK;
}

int read_status(const Workspace& w, SolveStatus* out, cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(out, w.status, sizeof(SolveStatus), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  return DG_OK;
}

int flags_to_status(int flags) {
  if (flags & kFlagTimeout) return fail(DG_ERR_TIMEOUT, "a device-side wait hit its cap");
  if (flags & kFlagBreakdown) return fail(DG_ERR_NONFINITE, "CG breakdown (p.q not positive or not finite)");
  if (flags & kFlagNoconv) return fail(DG_ERR_NOCONV, "CG reached maxit before the tolerance");
  return DG_OK;
}

int finish_invariants(const Workspace& w, double out[3], cudaStream_t st) {
  CUDA_TRY(cudaMemcpyAsync(w.host_out, w.inv_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  for (int j = 0; j < 3; ++j) out[j] = w.host_out[j];
  for (int j = 0; j < 3; ++j)
    if (!std::isfinite(out[j])) return fail(DG_ERR_NONFINITE, "invariant %d is not finite", j);
  return DG_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------------------

extern "C" {

const char* dg_last_error(void) { return g_err; }

int dg_version(void) { return 100; }

int dg_selftest_wait_cap(void* stream) {
  cudaStream_t st = as_stream(stream);
  SyncState* s = nullptr;
  int* out = nullptr;
  CUDA_TRY(cudaMalloc(&s, sizeof(SyncState)));
  CUDA_TRY(cudaMalloc(&out, sizeof(int)));
  CUDA_TRY(cudaMemsetAsync(s, 0, sizeof(SyncState), st));
  CUDA_TRY(cudaMemsetAsync(out, 0, sizeof(int), st));
  cudaError_t e = launch_barrier_selftest(s, out, st);
  int flags = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&flags, out, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(s);
  cudaFree(out);
  if (e != cudaSuccess) return fail(DG_ERR_CUDA, "self-test launch failed: %s", cudaGetErrorString(e));
  return (flags & kFlagTimeout) ? fail(DG_ERR_TIMEOUT, "device-side wait gave up as designed") : DG_OK;
}

int dg_ref_tables_len(int n) { return (n >= 1 && n <= kMaxN) ? 7 * n + 2 * n * n : 0; }

int dg_ref_tables(int n, double tau, double* out, int out_len) {
  if (n < 1 || n > kMaxN) return fail(DG_ERR_ARG, "n = %d outside 1..5", n);
  if (!(tau >= 0.0)) return fail(DG_ERR_ARG, "tau must be >= 0");
  if (!out || out_len < dg_ref_tables_len(n)) return fail(DG_ERR_ARG, "output buffer too small");
  RefTables t;
  if (build_ref_tables(n, tau, &t)) return fail(DG_ERR_ARG, "table construction failed");
  double* o = out;
  for (int i = 0; i < n; ++i) *o++ = t.x[i];
  for (int i = 0; i < n; ++i) *o++ = t.w[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) *o++ = t.C0[i][j];
  for (int i = 0; i < n; ++i) *o++ = t.muR[i];
  for (int i = 0; i < n; ++i) *o++ = t.muL[i];
  for (int i = 0; i < n; ++i) *o++ = t.lL[i];
  for (int i = 0; i < n; ++i) *o++ = t.lR[i];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) *o++ = t.A1cc[i][j];
  for (int i = 0; i < n; ++i) *o++ = t.betaA[i];
  return DG_OK;
}

int dg_grid_create(dg_grid** gp, int Nx, int Ny, int n, double Lx, double Ly, double tau) {
  return dg_grid_create_bc(gp, Nx, Ny, n, Lx, Ly, tau, DG_BC_PERIODIC);
}

int dg_grid_create_bc(dg_grid** gp, int Nx, int Ny, int n, double Lx, double Ly, double tau, int bc) {
  if (!gp) return fail(DG_ERR_ARG, "g is NULL");
  *gp = nullptr;
  if (bc != DG_BC_PERIODIC && bc != DG_BC_DIRICHLET) return fail(DG_ERR_ARG, "unknown boundary condition %d", bc);
  if (bc == DG_BC_DIRICHLET && tau != 0.0) return fail(DG_ERR_ARG, "Dirichlet grids take no jump penalty (tau = 0)");
  if (n < 1 || n > kMaxN) return fail(DG_ERR_ARG, "n = %d outside 1..5", n);
  if (Nx < 1 || Ny < 1) return fail(DG_ERR_ARG, "Nx, Ny must be >= 1");
  if ((long long)Nx * Ny * n * n > (1ll << 31)) return fail(DG_ERR_ARG, "grid too large");
  if (!(Lx > 0.0) || !(Ly > 0.0)) return fail(DG_ERR_ARG, "Lx, Ly must be > 0");
  if (!(tau >= 0.0)) return fail(DG_ERR_ARG, "tau must be >= 0");
  dg_grid* g = new (std::nothrow) dg_grid();
  if (!g) return fail(DG_ERR_NOMEM, "host allocation failed");
  g->Nx = Nx;
  g->Ny = Ny;
  g->n = n;
  g->Lx = Lx;
  g->Ly = Ly;
  g->hx = Lx / Nx;
  g->hy = Ly / Ny;
  g->tau = tau;
  g->bc = bc;
  build_ref_tables(n, tau, &g->rt);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete g;
    return fail(DG_ERR_CUDA, "no CUDA device: %s", cudaGetErrorString(e));
  }
  choose_tiles(n, Nx, Ny, g->num_sms, g->rTY, g->rTX, g->cTY, g->cTX);
  dispatch_n(n, [&](auto nc) {
    build_ops<decltype(nc)::value>(g);
    return DG_OK;
  });
  int rc = alloc_ws(g->ws, ndof_of(g), co_resident_cap(g), true);
  if (!rc) rc = alloc_ws_precond(g->ws, Nx, Ny, n, false);
  if (!rc) rc = build_pc(g);
  if (!rc) rc = upload_ops(g);
  if (rc) {
    free_ws(g->ws);
    free_pc(g->pc);
    delete g;
    return rc;
  }
  *gp = g;
  return DG_OK;
}

int dg_grid_destroy(dg_grid* g) {
  if (!g) return DG_OK;
  free_ws(g->ws);
  free_pc(g->pc);
  cudaFree(g->d_opsd);
  cudaFree(g->d_opsf);
  cudaFree(g->d_opsx);
  cudaFree(g->d_opsk);
  delete g;
  return DG_OK;
}

int dg_grid_set_compensated_apply(dg_grid* g, int mode) {
  if (!g) return fail(DG_ERR_ARG, "g is NULL");
  if (mode < -1 || mode > 2) return fail(DG_ERR_ARG, "mode must be -1 (automatic), 0, 1 or 2");
  g->precise_apply = mode < 0 ? g->precise_auto : mode;
  return DG_OK;
}

int dg_grid_get_compensated_apply(const dg_grid* g) { return g ? g->precise_apply : 0; }

constexpr int kSpectralDirectMax = 256;  // longest non-power-of-two line of the spectral DFTs

int dg_grid_set_precond(dg_grid* g, int kind) {
  if (!g) return fail(DG_ERR_ARG, "g is NULL");
  if (kind != DG_PRECOND_JACOBI && kind != DG_PRECOND_TWOLEVEL && kind != DG_PRECOND_SPECTRAL)
    return fail(DG_ERR_ARG, "unknown preconditioner %d", kind);
  if (kind == DG_PRECOND_TWOLEVEL && g->bc != DG_BC_PERIODIC)
    return fail(DG_ERR_ARG, "the two-level preconditioner's coarse DFT solve needs a periodic grid");
  if (kind == DG_PRECOND_SPECTRAL && g->bc != DG_BC_PERIODIC)
    return fail(DG_ERR_ARG, "the spectral preconditioner needs a periodic grid");
  if (kind == DG_PRECOND_SPECTRAL && g->pc.spectral_rc != DG_OK)
    return fail(DG_ERR_ARG, "the spectral preconditioner's tables could not be built for this grid");
  // a side that is not a power of two takes the direct O(L^2) DFT per line: fine for small
  // lines, far slower than CG with another preconditioner beyond a few hundred cells
  if (kind == DG_PRECOND_SPECTRAL && ((g->pc.log2x < 0 && g->Nx > kSpectralDirectMax) ||
                                      (g->pc.log2y < 0 && g->Ny > kSpectralDirectMax)))
    return fail(DG_ERR_ARG, "the spectral preconditioner needs cell counts that are powers of two above %d",
                kSpectralDirectMax);
  g->precond = kind;
  return DG_OK;
}

int dg_spectral_symbol(int N, int n, double L, double tau, int k, double* lam, double* Vre, double* Vim) {
  if (n < 1 || n > kMaxN) return fail(DG_ERR_ARG, "n = %d outside 1..5", n);
  if (N < 1 || k < 0 || k >= N || !(L > 0.0) || !(tau >= 0.0)) return fail(DG_ERR_ARG, "bad line or wave number");
  if (!lam || !Vre || !Vim) return fail(DG_ERR_ARG, "NULL argument");
  RefTables t;
  if (build_ref_tables(n, tau, &t)) return fail(DG_ERR_ARG, "table construction failed");
  return dispatch_n(n, [&](auto nc) {
    constexpr int NC = decltype(nc)::value;
    const Ops2D<double, NC> O = make_ops<double, NC>(t, L / N, L / N);
    return spectral_symbol<NC>(O.kx, N, k, lam, Vre, Vim);
  });
}

long long dg_grid_dof(const dg_grid* g) { return g ? (long long)ndof_of(g) : 0; }

int dg_grid_nodes(const dg_grid* g, double* xn, double* yn, double* w) {
  if (!g) return fail(DG_ERR_ARG, "g is NULL");
  const int n = g->n;
  if (xn)
    for (int c = 0; c < g->Nx; ++c)
      for (int b = 0; b < n; ++b) xn[c * n + b] = (c + 0.5) * g->hx + 0.5 * g->hx * g->rt.x[b];
  if (yn)
    for (int c = 0; c < g->Ny; ++c)
      for (int a = 0; a < n; ++a) yn[c * n + a] = (c + 0.5) * g->hy + 0.5 * g->hy * g->rt.x[a];
  if (w)
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) w[a * n + b] = (g->hy * 0.5 * g->rt.w[a]) * (g->hx * 0.5 * g->rt.w[b]);
  return DG_OK;
}

int dg_grid_set_tiles(dg_grid* g, int TY, int TX) {
  if (!g) return fail(DG_ERR_ARG, "g is NULL");
  if (TY == 0 && TX == 0) {
    choose_tiles(g->n, g->Nx, g->Ny, g->num_sms, g->rTY, g->rTX, g->cTY, g->cTX);
    return DG_OK;
  }
  if (TY < 1 || TX < 1 || TY > 64 || TX > 64) return fail(DG_ERR_ARG, "tile must be 1..64 cells per side");
  const size_t rs = (size_t)(TY + 2) * (TX + 2) * (7 * (g->n * g->n + 1) + 12 * g->n) * sizeof(double);
  if (rs > 200 * 1024) return fail(DG_ERR_ARG, "tile %dx%d needs %zu B of shared memory", TY, TX, rs);
  g->rTY = g->cTY = TY;
  g->rTX = g->cTX = TX;
  return DG_OK;
}

int dg_bracket(dg_grid* g, const double* psi, const double* omega, double* J, void* stream) {
  if (!g || !psi || !omega || !J) return fail(DG_ERR_ARG, "NULL argument");
  if (!aligned8(psi) || !aligned8(omega) || !aligned8(J)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (J == psi || J == omega) return fail(DG_ERR_ARG, "J must not alias psi or omega");
  RhsArgs<double> A{};
  A.psi = psi;
  A.omega_in = omega;
  A.omega_base = omega;
  A.omega_out = J;
  A.bracket_only = 1;
  return dispatch_n(g->n, [&](auto nc) { return launch_rhs<double, decltype(nc)::value>(g, A, as_stream(stream)); });
}

int dg_bracket_parts(dg_grid* g, const double* psi, const double* omega, double* J, int parts, void* stream) {
  if (!g || !psi || !omega || !J) return fail(DG_ERR_ARG, "NULL argument");
  if (parts < 1 || parts > 7) return fail(DG_ERR_ARG, "parts must be a non-empty subset of {1, 2, 4}");
  if (!aligned8(psi) || !aligned8(omega) || !aligned8(J)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (J == psi || J == omega) return fail(DG_ERR_ARG, "J must not alias psi or omega");
  RhsArgs<double> A{};
  A.psi = psi;
  A.omega_in = omega;
  A.omega_base = omega;
  A.omega_out = J;
  A.bracket_only = 1;
  A.parts = parts;
  return dispatch_n(g->n, [&](auto nc) { return launch_rhs<double, decltype(nc)::value>(g, A, as_stream(stream)); });
}

int dg_bracket_mixed(dg_grid* g, const double* psi, const double* omega, double* J, void* stream) {
  if (!g || !psi || !omega || !J) return fail(DG_ERR_ARG, "NULL argument");
  if (!aligned8(psi) || !aligned8(omega) || !aligned8(J)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (J == psi || J == omega) return fail(DG_ERR_ARG, "J must not alias psi or omega");
  RhsArgs<df> A{};
  A.psi = psi;
  A.omega_in = omega;
  A.omega_base = omega;
  A.omega_out = J;
  A.bracket_only = 1;
  return dispatch_n(g->n, [&](auto nc) { return launch_rhs<df, decltype(nc)::value>(g, A, as_stream(stream)); });
}

int dg_laplace_apply(dg_grid* g, const double* x, double* y, int mode, void* stream) {
  if (!g || !x || !y) return fail(DG_ERR_ARG, "NULL argument");
  if (mode != 0 && mode != 1) return fail(DG_ERR_ARG, "mode must be 0 (A x) or 1 (Delta_h x)");
  if (!aligned8(x) || !aligned8(y)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (x == y) return fail(DG_ERR_ARG, "y must not alias x");
  return dispatch_n(g->n,
                    [&](auto nc) { return launch_apply<double, decltype(nc)::value>(g, x, y, mode, as_stream(stream)); });
}

int dg_poisson_solve(dg_grid* g, const double* omega, double* psi, double tol, int maxit, int fixed_iters,
                     int* iters, double* relres, void* stream) {
  if (!g || !omega || !psi) return fail(DG_ERR_ARG, "NULL argument");
  if (!aligned8(omega) || !aligned8(psi)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (maxit < 0 || fixed_iters < 0) return fail(DG_ERR_ARG, "maxit and fixed_iters must be >= 0");
  if (fixed_iters == 0 && !(tol > 0.0)) return fail(DG_ERR_ARG, "tol must be > 0");
  cudaStream_t st = as_stream(stream);
  CgArgs<double> A{};
  A.omega = omega;
  A.xa = psi;
  A.ca = 1.0;
  A.x_unscaled = 1;
  A.v = CgVectors<double>{g->ws.y, g->ws.r, g->ws.p0, g->ws.p1, g->ws.q};
  A.precond = g->precond;
  A.psi_out = psi;
  A.tol2 = tol * tol;
  A.floor2 = g->floor2;
  A.keep_mean = g->bc;
  A.maxit = fixed_iters > 0 ? std::max(maxit, fixed_iters) : maxit;
  A.fixed_iters = fixed_iters;
  A.sumW = g->Lx * g->Ly;
  int rc = dispatch_n(g->n, [&](auto nc) { return launch_cg<double, decltype(nc)::value>(g, A, g->ws, st); });
  if (rc) return rc;
  SolveStatus s;
  if ((rc = read_status(g->ws, &s, st))) return rc;
  if (iters) *iters = s.last_iters;
  if (relres) *relres = s.last_rhob > 0 ? std::sqrt(std::max(s.last_rho, 0.0) / s.last_rhob) : 0.0;
  return flags_to_status(s.last_flags);
}

int dg_invariants(dg_grid* g, const double* psi, const double* omega, double out[3], void* stream) {
  if (!g || !psi || !omega || !out) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  int rc = dispatch_n(g->n, [&](auto nc) {
    return launch_invariants<decltype(nc)::value>(g, psi, omega, 0, g->ws, st);
  });
  if (rc) return rc;
  return finish_invariants(g->ws, out, st);
}

// ---------------------------------------------------------------------------------------
// Simulations
// ---------------------------------------------------------------------------------------

}  // extern "C"

namespace {

void free_events(dg_sim* s) {
  for (auto e : s->ev_rhs) cudaEventDestroy(e);
  for (auto e : s->ev_cg) cudaEventDestroy(e);
  s->ev_rhs.clear();
  s->ev_cg.clear();
  s->n_ev_rhs = s->n_ev_cg = 0;
}

void free_sim(dg_sim* s) {
  free_events(s);
  for (auto& p : s->omega) cudaFree(p);
  for (auto& p : s->psi) cudaFree(p);
  for (auto& p : s->apsi) cudaFree(p);
  for (auto& p : s->R) cudaFree(p);
  cudaFree(s->stA);
  cudaFree(s->stB);
  cudaFree(s->k2);
  cudaFree(s->k3);
  free_ws(s->ws);
}

// Poisson solve inside the stepper: y = solve(omega) from y0 = ca xa + cb xb (scaled space):
// the persistent float64 CG kernel, or (DG_MIXED, DG_MIXED64) the float64-residual /
// float32-CG refinement kernel.
int sim_solve(dg_sim* s, const double* omega, const double* xa, double ca, const double* xb, double cb, double* y,
              cudaStream_t st, const double* axa = nullptr, const double* axb = nullptr, double* ay = nullptr) {
  dg_grid* g = s->g;
  int rc;
  if (s->fixed_iters > 0) axa = axb = ay = nullptr;  // parity mode: the plain operator applications
  if (s->precision == DG_FP64_PC32) {
    CgArgs<double, float> A{};
    A.omega = omega;
    A.xa = xa;
    A.xb = xb;
    A.ca = ca;
    A.cb = cb;
    A.x_unscaled = 0;
    A.axa = axa;
    A.axb = axb;
    A.ay = ay;
    A.v = CgVectors<double>{y, s->ws.r, s->ws.p0, s->ws.p1, s->ws.q};
    A.precond = g->precond;
    A.tol2 = s->tol * s->tol;
    A.floor2 = g->floor2;
    A.keep_mean = g->bc;
    A.maxit = s->fixed_iters > 0 ? std::max(s->maxit, s->fixed_iters) : s->maxit;
    A.fixed_iters = s->fixed_iters;
    A.sumW = g->Lx * g->Ly;
    rc = dispatch_n(g->n, [&](auto nc) { return launch_cg<double, decltype(nc)::value, float>(g, A, s->ws, st, s); });
  } else if (s->precision != DG_FP64) {
    MixedArgs A{};
    A.omega = omega;
    A.xa = xa;
    A.xb = xb;
    A.ca = ca;
    A.cb = cb;
    A.x_unscaled = 0;
    A.axa = axa;
    A.axb = axb;
    A.ay = ay;
    A.y = y;
    A.precond = g->precond;
    A.tol2 = s->tol * s->tol;
    A.floor2 = g->floor2;
    A.keep_mean = g->bc;
    A.tol_in2 = s->tol_in * s->tol_in;
    A.max_sweeps = s->max_sweeps;
    A.maxit_in = s->maxit;
    A.sumW = g->Lx * g->Ly;
    A.precise_apply = g->precise_apply;
    rc = dispatch_n(g->n, [&](auto nc) { return launch_mixed<decltype(nc)::value>(g, A, s->ws, st, s); });
  } else {
    CgArgs<double> A{};
    A.omega = omega;
    A.xa = xa;
    A.xb = xb;
    A.ca = ca;
    A.cb = cb;
    A.x_unscaled = 0;
    A.axa = axa;
    A.axb = axb;
    A.ay = ay;
    A.v = CgVectors<double>{y, s->ws.r, s->ws.p0, s->ws.p1, s->ws.q};
    A.precond = g->precond;
    A.tol2 = s->tol * s->tol;
    A.floor2 = g->floor2;
    A.keep_mean = g->bc;
    A.maxit = s->fixed_iters > 0 ? std::max(s->maxit, s->fixed_iters) : s->maxit;
    A.fixed_iters = s->fixed_iters;
    A.sumW = g->Lx * g->Ly;
    rc = dispatch_n(g->n, [&](auto nc) { return launch_cg<double, decltype(nc)::value>(g, A, s->ws, st, s); });
  }
  if (!rc) {
    s->launches += 1;
    s->cg_launches += 1;
  }
  return rc;
}

// R = -J(psi, omega_in) + D Delta_h omega_in;  omega_out = omega_base + dt (c_new R + sum c_m hist_m).
// R and the history are float64; the RHS is evaluated in float64 or, for DG_MIXED, in
// double-float arithmetic on the float32 pipe.
template <typename T>
int sim_rhs_t(dg_sim* s, const double* psi, const double* om_in, const double* om_base, double* om_out, void* R_out,
              double c_new, int nhist, void* const* hist, const double* c_hist, cudaStream_t st) {
  RhsArgs<T> A{};
  A.psi = psi;
  A.omega_in = om_in;
  A.omega_base = om_base;
  A.omega_out = om_out;
  A.R_out = static_cast<hist_t<T>*>(R_out);
  A.c_new = c_new;
  A.nhist = nhist;
  for (int m = 0; m < nhist; ++m) {
    A.hist[m] = static_cast<const hist_t<T>*>(hist[m]);
    A.c_hist[m] = c_hist[m];
  }
  A.dt = s->dt;
  A.visc = s->D;
  A.psi_scaled = 1;
  A.parts = s->parts;
  return dispatch_n(s->g->n, [&](auto nc) { return launch_rhs<T, decltype(nc)::value>(s->g, A, st); });
}

int sim_rhs(dg_sim* s, const double* psi, const double* om_in, const double* om_base, double* om_out, void* R_out,
            double c_new, int nhist, void* const* hist, const double* c_hist, cudaStream_t st) {
  int rc;
  if (s->timing && (rc = record_event(s->ev_rhs, s->n_ev_rhs, st))) return rc;
  rc = (s->precision == DG_MIXED)
           ? sim_rhs_t<df>(s, psi, om_in, om_base, om_out, R_out, c_new, nhist, hist, c_hist, st)
           : sim_rhs_t<double>(s, psi, om_in, om_base, om_out, R_out, c_new, nhist, hist, c_hist, st);
  if (rc) return rc;
  if (s->timing && (rc = record_event(s->ev_rhs, s->n_ev_rhs, st))) return rc;
  s->launches += 1;
  s->rhs_launches += 1;
  return DG_OK;
}

// R^k (just written into the free slot) becomes R^{k-1} of the next step; the oldest slot
// is freed: (r1, r2, r3, free) <- (free, r1, r2, r3).
void rotate_history(dg_sim* s) {
  const int r1 = s->r1, r2 = s->r2, r3 = s->r3, rf = s->rfree;
  s->r1 = rf;
  s->r2 = r1;
  s->r3 = r2;
  s->rfree = r3;
}

// Adams-Bashforth weights of R^k, R^{k-1}, ... for K = 1..4.
const double kAB[5][4] = {{0, 0, 0, 0},
                          {1.0, 0, 0, 0},
                          {3.0 / 2.0, -1.0 / 2.0, 0, 0},
                          {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0},
                          {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0}};

// A stepper solve into psi slot `out` from the guess ca psi[a] + cb psi[b] (b < 0: none),
// recycling the slots' operator products when they are known and keeping the result's.
int sim_solve_slots(dg_sim* s, const double* omega, int a, double ca, int b, double cb, int out, cudaStream_t st) {
  const bool rec = s->fixed_iters == 0 && s->apsi_ok[a] && (b < 0 || s->apsi_ok[b]);
  s->apsi_ok[out] = false;
  const int rc = sim_solve(s, omega, s->psi[a], ca, b < 0 ? nullptr : s->psi[b], cb, s->psi[out], st,
                           rec ? s->apsi[a] : nullptr, rec && b >= 0 ? s->apsi[b] : nullptr, s->apsi[out]);
  if (!rc) s->apsi_ok[out] = s->fixed_iters == 0;
  return rc;
}

// One classical RK4 step (start-up of the multistep method).  k1 is kept as R^k.
int sim_rk4_step(dg_sim* s, cudaStream_t st) {
  const double* w0 = s->omega[s->oc];
  double* w1 = s->omega[s->oc ^ 1];
  void* k1 = s->R[s->rfree];
  const int sA = s->p2, sB = s->p1;
  double* PA = s->psi[sA];
  double* PB = s->psi[sB];
  const double* P0 = s->psi[s->p0];
  int rc;
  if ((rc = sim_rhs(s, P0, w0, w0, s->stA, k1, 0.5, 0, nullptr, nullptr, st))) return rc;
  if ((rc = sim_solve_slots(s, s->stA, s->p0, 1.0, -1, 0.0, sA, st))) return rc;
  if ((rc = sim_rhs(s, PA, s->stA, w0, s->stB, s->k2, 0.5, 0, nullptr, nullptr, st))) return rc;
  if ((rc = sim_solve_slots(s, s->stB, sA, 1.0, -1, 0.0, sB, st))) return rc;
  if ((rc = sim_rhs(s, PB, s->stB, w0, s->stA, s->k3, 1.0, 0, nullptr, nullptr, st))) return rc;
  if ((rc = sim_solve_slots(s, s->stA, sB, 1.0, -1, 0.0, sA, st))) return rc;
  void* const hist[3] = {k1, s->k2, s->k3};
  const double ch[3] = {1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0};
  if ((rc = sim_rhs(s, PA, s->stA, w0, w1, nullptr, 1.0 / 6.0, 3, hist, ch, st))) return rc;
  if ((rc = sim_solve_slots(s, w1, sA, 1.0, -1, 0.0, sB, st))) return rc;
  // psi^{k+1} = PB (old p1 slot), psi^k stays p0: rotate (p0, p1, p2) <- (p1, p0, p2)
  std::swap(s->p0, s->p1);
  rotate_history(s);
  s->oc ^= 1;
  s->step += 1;
  return DG_OK;
}

// One Adams-Bashforth step of order K (K = 3 in the paper's runs):
//   omega^{k+1} = omega^k + dt sum_m beta_m R^{k-m},
// then the Poisson solve from the extrapolation 2 psi^k - psi^{k-1}.
int sim_ab3_step(dg_sim* s, cudaStream_t st) {
  const double* w0 = s->omega[s->oc];
  double* w1 = s->omega[s->oc ^ 1];
  void* Rk = s->R[s->rfree];
  void* const hist[3] = {s->R[s->r1], s->R[s->r2], s->R[s->r3]};
  const int K = s->K;
  const double ch[3] = {kAB[K][1], kAB[K][2], kAB[K][3]};
  int rc;
  if ((rc = sim_rhs(s, s->psi[s->p0], w0, w0, w1, Rk, kAB[K][0], K - 1, hist, ch, st))) return rc;
  if ((rc = sim_solve_slots(s, w1, s->p0, 2.0, s->p1, -1.0, s->p2, st))) return rc;
  const int np0 = s->p2, np1 = s->p0, np2 = s->p1;
  s->p0 = np0;
  s->p1 = np1;
  s->p2 = np2;
  rotate_history(s);
  s->oc ^= 1;
  s->step += 1;
  return DG_OK;
}

// History buffer <-> float64 device array.
int R_to_double(const dg_sim* s, const void* R, double* dst, cudaStream_t st) {
  const size_t nd = ndof_of(s->g);
  CUDA_TRY(cudaMemcpyAsync(dst, R, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return DG_OK;
}

int R_from_double(const dg_sim* s, const double* src, void* R, cudaStream_t st) {
  const size_t nd = ndof_of(s->g);
  CUDA_TRY(cudaMemcpyAsync(R, src, nd * sizeof(double), cudaMemcpyDeviceToDevice, st));
  return DG_OK;
}

int scale_field(const dg_grid* g, const double* x, double* y, int inverse, cudaStream_t st) {
  return dispatch_n(g->n, [&](auto nc) { return launch_scale<decltype(nc)::value>(g, x, y, inverse, st); });
}

}  // namespace

extern "C" {

}  // extern "C"

namespace {

// Layout of a dg_sim_save file: this header, then six arrays of Nx Ny n^2 float64 values in the
// cell-blocked node order (omega^k, sqrt(W) psi^k, sqrt(W) psi^{k-1}, R^{k-1}, R^{k-2},
// R^{k-3}); little-endian, as written by the host.
const char kSimMagic[8] = {'D', 'G', 'S', 'I', 'M', '0', '0', '2'};
struct SimFileHeader {
  char magic[8];
  int32_t Nx, Ny, n, precision;
  int32_t K, bracket, maxit, fixed_iters;
  int32_t max_sweeps, precond;
  int64_t step;
  double Lx, Ly, tau, D, dt, tol, tol_in;
  int32_t bc, reserved;
};
static_assert(sizeof(SimFileHeader) == 120, "file header layout");

// A simulation with all its buffers allocated and no state yet (step 0, rings at rest).
int sim_new(dg_sim** sp, dg_grid* g, double D, double dt, int precision, double cg_tol, int cg_maxit) {
  *sp = nullptr;
  if (!(D >= 0.0) || !(dt > 0.0) || !(cg_tol > 0.0) || cg_maxit < 1)
    return fail(DG_ERR_ARG, "need D >= 0, dt > 0, cg_tol > 0, cg_maxit >= 1");
  if (precision != DG_FP64 && precision != DG_MIXED && precision != DG_MIXED64 && precision != DG_FP64_PC32)
    return fail(DG_ERR_ARG, "unknown precision %d", precision);
  dg_sim* s = new (std::nothrow) dg_sim();
  if (!s) return fail(DG_ERR_NOMEM, "host allocation failed");
  s->g = g;
  s->D = D;
  s->dt = dt;
  s->tol = cg_tol;
  s->maxit = cg_maxit;
  s->precision = precision;
  s->tol_in = 1e-4;
  s->max_sweeps = 40;
  s->p0 = 0;
  s->p1 = 1;
  s->p2 = 2;
  s->r1 = 0;
  s->r2 = 1;
  s->r3 = 2;
  s->rfree = 3;
  const size_t bytes = ndof_of(g) * sizeof(double);
  const size_t rbytes = ndof_of(g) * sizeof(double);
  auto alloc_all = [&]() -> int {
    for (auto& p : s->omega) CUDA_TRY(cudaMalloc(&p, bytes));
    for (auto& p : s->psi) CUDA_TRY(cudaMalloc(&p, bytes));
    for (auto& p : s->apsi) CUDA_TRY(cudaMalloc(&p, bytes));
    for (auto& p : s->R) CUDA_TRY(cudaMalloc(&p, rbytes));
    CUDA_TRY(cudaMalloc(&s->stA, bytes));
    CUDA_TRY(cudaMalloc(&s->stB, bytes));
    CUDA_TRY(cudaMalloc(&s->k2, rbytes));
    CUDA_TRY(cudaMalloc(&s->k3, rbytes));
    if (int rc = alloc_ws(s->ws, ndof_of(g), co_resident_cap(g), false)) return rc;
    if (int rc = alloc_ws_precond(s->ws, g->Nx, g->Ny, g->n, precision != DG_FP64)) return rc;
    return (precision == DG_MIXED || precision == DG_MIXED64) ? alloc_ws_mixed(s->ws) : DG_OK;
  };
  if (int rc = alloc_all()) {
    free_sim(s);
    delete s;
    return rc;
  }
  *sp = s;
  return DG_OK;
}

}  // namespace

extern "C" {

int dg_sim_create(dg_sim** sp, dg_grid* g, double D, double dt, int precision, double cg_tol, int cg_maxit,
                  const double* omega0, void* stream) {
  if (!sp) return fail(DG_ERR_ARG, "s is NULL");
  *sp = nullptr;
  if (!g || !omega0) return fail(DG_ERR_ARG, "NULL argument");
  if (!aligned8(omega0)) return fail(DG_ERR_ARG, "misaligned pointer");
  cudaStream_t st = as_stream(stream);
  dg_sim* s = nullptr;
  if (int rc = sim_new(&s, g, D, dt, precision, cg_tol, cg_maxit)) return rc;
  const size_t bytes = ndof_of(g) * sizeof(double);
  int rc = (cudaMemcpyAsync(s->omega[0], omega0, bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess)
                    ? DG_OK
                    : fail(DG_ERR_CUDA, "copy of omega0 failed");
  // psi^0 from a zero initial guess; psi^{-1} = psi^0 so the first extrapolation is psi^0.
  if (!rc) rc = sim_solve(s, s->omega[0], nullptr, 0.0, nullptr, 0.0, s->psi[0], st, nullptr, nullptr, s->apsi[0]);
  if (!rc && (cudaMemcpyAsync(s->psi[1], s->psi[0], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
              cudaMemcpyAsync(s->apsi[1], s->apsi[0], bytes, cudaMemcpyDeviceToDevice, st) != cudaSuccess))
    rc = fail(DG_ERR_CUDA, "copy failed");
  s->apsi_ok[0] = s->apsi_ok[1] = !rc;
  SolveStatus ss;
  if (!rc) rc = read_status(s->ws, &ss, st);
  if (!rc) rc = flags_to_status(ss.last_flags);
  if (rc) {
    free_sim(s);
    delete s;
    return rc;
  }
  *sp = s;
  return DG_OK;
}

int dg_sim_destroy(dg_sim* s) {
  if (!s) return DG_OK;
  free_sim(s);
  delete s;
  return DG_OK;
}

int dg_step(dg_sim* s, int nsteps, void* stream) {
  if (!s || nsteps < 0) return fail(DG_ERR_ARG, "bad arguments");
  cudaStream_t st = as_stream(stream);
  for (int i = 0; i < nsteps; ++i) {
    const int rc = (s->step < s->K - 1) ? sim_rk4_step(s, st) : sim_ab3_step(s, st);
    if (rc) return rc;
  }
  return DG_OK;
}

int dg_sim_status(dg_sim* s, dg_sim_info* info, void* stream) {
  if (!s || !info) return fail(DG_ERR_ARG, "NULL argument");
  SolveStatus ss;
  if (int rc = read_status(s->ws, &ss, as_stream(stream))) return rc;
  info->step = s->step;
  info->cg_iters_total = ss.total_iters;
  info->cg_iters_last = ss.last_iters;
  info->cg_iters_max = ss.max_iters;
  info->cg_relres_last = ss.last_rhob > 0 ? std::sqrt(std::max(ss.last_rho, 0.0) / ss.last_rhob) : 0.0;
  info->refine_sweeps_last = ss.last_sweeps;
  info->status = ss.flags ? flags_to_status(ss.flags) : DG_OK;
  return info->status;
}

int dg_sim_refinement_history(dg_sim* s, double* relres, int* inner_iters, int max, int* count, void* stream) {
  if (!s || !count || max < 0 || (max > 0 && (!relres || !inner_iters))) return fail(DG_ERR_ARG, "bad arguments");
  SolveStatus ss;
  if (int rc = read_status(s->ws, &ss, as_stream(stream))) return rc;
  const int len = std::min(ss.hist_len, kRefineHistory);
  *count = len;
  for (int j = 0; j < len && j < max; ++j) {
    relres[j] = std::sqrt(std::max(ss.hist_rr[j], 0.0));
    inner_iters[j] = (j + 1 < len || ss.last_sweeps > j) ? ss.hist_it[j] : 0;
  }
  return DG_OK;
}

int dg_sim_get(dg_sim* s, double* omega, double* psi, void* stream) {
  if (!s) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = ndof_of(s->g) * sizeof(double);
  if (omega) CUDA_TRY(cudaMemcpyAsync(omega, s->omega[s->oc], bytes, cudaMemcpyDeviceToDevice, st));
  if (psi) return scale_field(s->g, s->psi[s->p0], psi, 1, st);
  return DG_OK;
}

int dg_sim_get_state(dg_sim* s, long long* step, double* omega, double* psi, double* psi_prev, double* R1, double* R2,
                     void* stream) {
  if (!s || !step || !omega || !psi || !psi_prev || !R1 || !R2) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = ndof_of(s->g) * sizeof(double);
  *step = s->step;
  CUDA_TRY(cudaMemcpyAsync(omega, s->omega[s->oc], bytes, cudaMemcpyDeviceToDevice, st));
  if (int rc = R_to_double(s, s->R[s->r1], R1, st)) return rc;
  if (int rc = R_to_double(s, s->R[s->r2], R2, st)) return rc;
  if (int rc = scale_field(s->g, s->psi[s->p0], psi, 1, st)) return rc;
  return scale_field(s->g, s->psi[s->p1], psi_prev, 1, st);
}

int dg_sim_set_state(dg_sim* s, long long step, const double* omega, const double* psi, const double* psi_prev,
                     const double* R1, const double* R2, void* stream) {
  if (!s || !omega || !psi || !psi_prev || !R1 || !R2 || step < 0) return fail(DG_ERR_ARG, "bad arguments");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = ndof_of(s->g) * sizeof(double);
  s->step = step;
  s->apsi_ok[0] = s->apsi_ok[1] = s->apsi_ok[2] = false;
  CUDA_TRY(cudaMemcpyAsync(s->omega[s->oc], omega, bytes, cudaMemcpyDeviceToDevice, st));
  if (int rc = R_from_double(s, R1, s->R[s->r1], st)) return rc;
  if (int rc = R_from_double(s, R2, s->R[s->r2], st)) return rc;
  if (int rc = scale_field(s->g, psi, s->psi[s->p0], 0, st)) return rc;
  return scale_field(s->g, psi_prev, s->psi[s->p1], 0, st);
}

int dg_sim_get_history(dg_sim* s, int m, double* R, void* stream) {
  if (!s || !R || m < 1 || m > 3) return fail(DG_ERR_ARG, "bad arguments");
  const int slot[3] = {s->r1, s->r2, s->r3};
  return R_to_double(s, s->R[slot[m - 1]], R, as_stream(stream));
}

int dg_sim_set_history(dg_sim* s, int m, const double* R, void* stream) {
  if (!s || !R || m < 1 || m > 3) return fail(DG_ERR_ARG, "bad arguments");
  const int slot[3] = {s->r1, s->r2, s->r3};
  return R_from_double(s, R, s->R[slot[m - 1]], as_stream(stream));
}

int dg_sim_set_cg(dg_sim* s, double tol, int maxit, int fixed_iters) {
  if (!s || !(tol > 0.0) || maxit < 1 || fixed_iters < 0) return fail(DG_ERR_ARG, "bad arguments");
  s->tol = tol;
  s->maxit = maxit;
  s->fixed_iters = fixed_iters;
  return DG_OK;
}

int dg_sim_upload(dg_sim* s, long long step, const double* omega, const double* psi, const double* psi_prev,
                  const double* R1, const double* R2, void* stream) {
  if (!s || !omega || !psi || !psi_prev || !R1 || !R2 || step < 0) return fail(DG_ERR_ARG, "bad arguments");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = ndof_of(s->g) * sizeof(double);
  s->step = step;
  CUDA_TRY(cudaMemcpyAsync(s->omega[s->oc], omega, bytes, cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(s->stA, R1, bytes, cudaMemcpyHostToDevice, st));
  if (int rc = R_from_double(s, s->stA, s->R[s->r1], st)) return rc;
  CUDA_TRY(cudaMemcpyAsync(s->stB, R2, bytes, cudaMemcpyHostToDevice, st));
  if (int rc = R_from_double(s, s->stB, s->R[s->r2], st)) return rc;
  CUDA_TRY(cudaMemcpyAsync(s->stA, psi, bytes, cudaMemcpyHostToDevice, st));
  if (int rc = scale_field(s->g, s->stA, s->psi[s->p0], 0, st)) return rc;
  CUDA_TRY(cudaMemcpyAsync(s->stB, psi_prev, bytes, cudaMemcpyHostToDevice, st));
  if (int rc = scale_field(s->g, s->stB, s->psi[s->p1], 0, st)) return rc;
  return DG_OK;
}

int dg_sim_download(dg_sim* s, double* omega, double* psi, void* stream) {
  if (!s) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  const size_t bytes = ndof_of(s->g) * sizeof(double);
  if (omega) CUDA_TRY(cudaMemcpyAsync(omega, s->omega[s->oc], bytes, cudaMemcpyDeviceToHost, st));
  if (psi) {
    if (int rc = scale_field(s->g, s->psi[s->p0], s->stA, 1, st)) return rc;
    CUDA_TRY(cudaMemcpyAsync(psi, s->stA, bytes, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return DG_OK;
}

int dg_sim_set_timing(dg_sim* s, int enable) {
  if (!s) return fail(DG_ERR_ARG, "NULL argument");
  s->timing = enable != 0;
  s->launches = s->rhs_launches = s->cg_launches = 0;
  s->n_ev_rhs = s->n_ev_cg = 0;
  return DG_OK;
}

int dg_sim_get_counters(dg_sim* s, dg_sim_counters* c, void* stream) {
  if (!s || !c) return fail(DG_ERR_ARG, "NULL argument");
  CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
  c->launches = s->launches;
  c->rhs_launches = s->rhs_launches;
  c->cg_launches = s->cg_launches;
  c->rhs_ms = c->cg_ms = 0.0;
  for (size_t i = 0; i + 1 < s->n_ev_rhs; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, s->ev_rhs[i], s->ev_rhs[i + 1]));
    c->rhs_ms += ms;
  }
  for (size_t i = 0; i + 1 < s->n_ev_cg; i += 2) {
    float ms = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms, s->ev_cg[i], s->ev_cg[i + 1]));
    c->cg_ms += ms;
  }
  return DG_OK;
}

int dg_sim_set_multistep(dg_sim* s, int K) {
  if (!s || K < 1 || K > 4) return fail(DG_ERR_ARG, "K must be in 1..4");
  s->K = K;
  return DG_OK;
}

int dg_sim_set_bracket(dg_sim* s, int variant) {
  if (!s || (variant != DG_BRACKET_ARAKAWA && variant != DG_BRACKET_NAIVE))
    return fail(DG_ERR_ARG, "unknown bracket variant");
  s->parts = variant == DG_BRACKET_NAIVE ? 1 : 0;
  return DG_OK;
}

int dg_sim_save(dg_sim* s, const char* path, void* stream) {
  if (!s || !path) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  const dg_grid* g = s->g;
  const size_t nd = ndof_of(g);
  SimFileHeader h{};
  std::memcpy(h.magic, kSimMagic, sizeof(h.magic));
  h.Nx = g->Nx;
  h.Ny = g->Ny;
  h.n = g->n;
  h.precision = s->precision;
  h.K = s->K;
  h.bracket = s->parts ? DG_BRACKET_NAIVE : DG_BRACKET_ARAKAWA;
  h.maxit = s->maxit;
  h.fixed_iters = s->fixed_iters;
  h.max_sweeps = s->max_sweeps;
  h.precond = g->precond;
  h.bc = g->bc;
  // reserved: bit 0 / 1 = the operator products of psi^k / psi^{k-1} follow the six fields
  h.reserved = (s->apsi_ok[s->p0] ? 1 : 0) | (s->apsi_ok[s->p1] ? 2 : 0);
  h.step = s->step;
  h.Lx = g->Lx;
  h.Ly = g->Ly;
  h.tau = g->tau;
  h.D = s->D;
  h.dt = s->dt;
  h.tol = s->tol;
  h.tol_in = s->tol_in;
  std::vector<double> host(nd);
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(DG_ERR_IO, "cannot open %s for writing", path);
  int rc = std::fwrite(&h, sizeof(h), 1, f) == 1 ? DG_OK : fail(DG_ERR_IO, "write failed");
  // omega, the solver variables sqrt(W) psi^k and sqrt(W) psi^{k-1}, then R^{k-1..k-3}, then
  // the known operator products Ahat psi^k, Ahat psi^{k-1} (reserved bits)
  const void* fields[8] = {s->omega[s->oc], s->psi[s->p0], s->psi[s->p1], s->R[s->r1], s->R[s->r2], s->R[s->r3],
                           s->apsi[s->p0], s->apsi[s->p1]};
  for (int i = 0; i < 8 && !rc; ++i) {
    if (i >= 6 && !(h.reserved & (1 << (i - 6)))) continue;
    const double* src = static_cast<const double*>(fields[i]);
    if (cudaMemcpyAsync(host.data(), src, nd * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
      rc = fail(DG_ERR_CUDA, "copy to the host failed");
      break;
    }
    if (std::fwrite(host.data(), sizeof(double), nd, f) != nd) rc = fail(DG_ERR_IO, "write failed");
  }
  if (std::fclose(f) != 0 && !rc) rc = fail(DG_ERR_IO, "close failed");
  return rc;
}

int dg_sim_load(dg_sim** sp, dg_grid* g, const char* path, void* stream) {
  if (!sp) return fail(DG_ERR_ARG, "s is NULL");
  *sp = nullptr;
  if (!g || !path) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(DG_ERR_IO, "cannot open %s", path);
  SimFileHeader h{};
  if (std::fread(&h, sizeof(h), 1, f) != 1 || std::memcmp(h.magic, kSimMagic, sizeof(h.magic)) != 0) {
    std::fclose(f);
    return fail(DG_ERR_IO, "%s is not a simulation file of this version", path);
  }
  if (h.Nx != g->Nx || h.Ny != g->Ny || h.n != g->n || h.Lx != g->Lx || h.Ly != g->Ly || h.tau != g->tau ||
      h.precond != g->precond || h.bc != g->bc) {
    std::fclose(f);
    return fail(DG_ERR_ARG, "the grid (size, n, domain, tau, preconditioner, boundaries) differs from the saved one");
  }
  if (h.K < 1 || h.K > 4 || h.step < 0 || (h.bracket != DG_BRACKET_ARAKAWA && h.bracket != DG_BRACKET_NAIVE) ||
      h.fixed_iters < 0 || h.max_sweeps < 1 || !(h.tol_in > 0.0 && h.tol_in < 1.0) || h.reserved < 0 ||
      h.reserved > 3) {
    std::fclose(f);
    return fail(DG_ERR_IO, "corrupt header in %s", path);
  }
  dg_sim* s = nullptr;
  if (int rc = sim_new(&s, g, h.D, h.dt, h.precision, h.tol, h.maxit)) {
    std::fclose(f);
    return rc;
  }
  s->K = h.K;
  s->parts = h.bracket == DG_BRACKET_NAIVE ? 1 : 0;
  s->fixed_iters = h.fixed_iters;
  s->max_sweeps = h.max_sweeps;
  s->tol_in = h.tol_in;
  s->step = h.step;
  const size_t nd = ndof_of(g);
  std::vector<double> host(nd);
  void* fields[8] = {s->omega[s->oc], s->psi[s->p0], s->psi[s->p1], s->R[s->r1], s->R[s->r2], s->R[s->r3],
                     s->apsi[s->p0], s->apsi[s->p1]};
  int rc = DG_OK;
  for (int i = 0; i < 8 && !rc; ++i) {
    if (i >= 6 && !(h.reserved & (1 << (i - 6)))) continue;
    if (std::fread(host.data(), sizeof(double), nd, f) != nd) {
      rc = fail(DG_ERR_IO, "%s is truncated", path);
      break;
    }
    double* dst = static_cast<double*>(fields[i]);
    if (cudaMemcpyAsync(dst, host.data(), nd * sizeof(double), cudaMemcpyHostToDevice, st) != cudaSuccess) {
      rc = fail(DG_ERR_CUDA, "copy to the device failed");
      break;
    }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = fail(DG_ERR_CUDA, "copy to the device failed");
  }
  std::fclose(f);
  if (rc) {
    free_sim(s);
    delete s;
    return rc;
  }
  s->apsi_ok[s->p0] = (h.reserved & 1) != 0;
  s->apsi_ok[s->p1] = (h.reserved & 2) != 0;
  *sp = s;
  return DG_OK;
}

int dg_sim_set_refinement(dg_sim* s, double tol_in, int max_sweeps) {
  if (!s || !(tol_in > 0.0) || !(tol_in < 1.0) || max_sweeps < 1) return fail(DG_ERR_ARG, "bad arguments");
  s->tol_in = tol_in;
  s->max_sweeps = max_sweeps;
  return DG_OK;
}

int dg_sim_invariants(dg_sim* s, double out[3], void* stream) {
  if (!s || !out) return fail(DG_ERR_ARG, "NULL argument");
  cudaStream_t st = as_stream(stream);
  int rc = dispatch_n(s->g->n, [&](auto nc) {
    return launch_invariants<decltype(nc)::value>(s->g, s->psi[s->p0], s->omega[s->oc], 1, s->ws, st);
  });
  if (rc) return rc;
  return finish_invariants(s->ws, out, st);
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Poisson solve without any allocation (dg_poisson_solve_static)
//
// For callers that cannot allocate device memory themselves -- code running where
// cudaMalloc is forbidden or unsafe, such as inside a CUDA stream capture that must not
// change the memory pool, or in a host process whose allocator is owned by another
// framework -- this entry point runs the same persistent CG kernel as dg_poisson_solve but
// keeps every scratch vector, the per-block partial sums, the grid barrier and the status
// word in one file-scope __device__ array of fixed size.  Each GPU that loads the library
// holds that array (about 2.8 MB) until the process exits.
// ---------------------------------------------------------------------------------------
namespace {

constexpr long long kStaticMaxDof = 65536;  // Nx * Ny * n * n accepted by the static solve
constexpr int kStaticMaxBlocks = 4096;      // cooperative blocks the partials can hold

struct StaticScratch {
  double y[kStaticMaxDof];
  double r[kStaticMaxDof];
  double p0[kStaticMaxDof];
  double p1[kStaticMaxDof];
  double q[kStaticMaxDof];
  double part[6 * kStaticMaxBlocks];
  SyncState sync;
  SolveStatus status;
};

static __device__ __align__(256) StaticScratch g_static_scratch;

// The array's name in host code is a host-side stand-in, not a device address.  Its device
// address on the current device is looked up at every call (cudaGetSymbolAddress allocates
// nothing and is cheap), so no address outlives a reset of the device's context.
int static_scratch_address(StaticScratch** out) {
  void* p = nullptr;
  CUDA_TRY(cudaGetSymbolAddress(&p, g_static_scratch));
  *out = static_cast<StaticScratch*>(p);
  return DG_OK;
}

}  // namespace

extern "C" int dg_poisson_solve_static(int Nx, int Ny, int n, double Lx, double Ly, double tau, const double* omega,
                                       double* psi, double tol, int maxit, int fixed_iters, int* iters,
                                       double* relres, void* stream) {
  if (n < 1 || n > kMaxN) return fail(DG_ERR_ARG, "n = %d outside 1..5", n);
  if (Nx < 1 || Ny < 1) return fail(DG_ERR_ARG, "Nx, Ny must be >= 1");
  if (!(Lx > 0.0) || !(Ly > 0.0) || !(tau >= 0.0)) return fail(DG_ERR_ARG, "need Lx, Ly > 0 and tau >= 0");
  const long long ndof = (long long)Nx * Ny * n * n;
  if (ndof > kStaticMaxDof)
    return fail(DG_ERR_ARG, "grid of %lld values exceeds the static scratch limit of %lld values (Nx*Ny*n*n)", ndof,
                kStaticMaxDof);
  if (!omega || !psi) return fail(DG_ERR_ARG, "NULL argument");
  if (!aligned8(omega) || !aligned8(psi)) return fail(DG_ERR_ARG, "misaligned pointer");
  if (maxit < 0 || fixed_iters < 0) return fail(DG_ERR_ARG, "maxit and fixed_iters must be >= 0");
  if (fixed_iters == 0 && !(tol > 0.0)) return fail(DG_ERR_ARG, "tol must be > 0");
  cudaStream_t st = as_stream(stream);
  StaticScratch* sc = nullptr;
  if (int rc = static_scratch_address(&sc)) return rc;

  // A grid description on the host stack, its workspace pointing into the static array.
  dg_grid g{};
  g.Nx = Nx;
  g.Ny = Ny;
  g.n = n;
  g.Lx = Lx;
  g.Ly = Ly;
  g.hx = Lx / Nx;
  g.hy = Ly / Ny;
  g.tau = tau;
  build_ref_tables(n, tau, &g.rt);
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&g.num_sms, cudaDevAttrMultiProcessorCount, dev));
  choose_tiles(n, Nx, Ny, g.num_sms, g.rTY, g.rTX, g.cTY, g.cTX);
  dispatch_n(n, [&](auto nc) {
    build_ops<decltype(nc)::value>(&g);
    return DG_OK;
  });
  Workspace w{};
  w.ndof = (size_t)ndof;
  w.grid_cap = kStaticMaxBlocks;
  w.y = sc->y;
  w.r = sc->r;
  w.p0 = sc->p0;
  w.p1 = sc->p1;
  w.q = sc->q;
  w.part = sc->part;
  w.sync = &sc->sync;
  w.status = &sc->status;
  // The status word accumulates across calls: start it at zero (the barrier state is
  // cleared by the launch itself).
  CUDA_TRY(cudaMemsetAsync(&sc->status, 0, sizeof(SolveStatus), st));

  CgArgs<double> A{};
  A.omega = omega;
  A.xa = psi;
  A.ca = 1.0;
  A.x_unscaled = 1;
  A.v = CgVectors<double>{w.y, w.r, w.p0, w.p1, w.q};
  A.psi_out = psi;
  A.tol2 = tol * tol;
  A.floor2 = g.floor2;
  A.maxit = fixed_iters > 0 ? std::max(maxit, fixed_iters) : maxit;
  A.fixed_iters = fixed_iters;
  A.sumW = Lx * Ly;
  int rc = dispatch_n(n, [&](auto nc) { return launch_cg<double, decltype(nc)::value>(&g, A, w, st); });
  if (rc) return rc;
  SolveStatus s;
  if ((rc = read_status(w, &s, st))) return rc;
  if (iters) *iters = s.last_iters;
  if (relres) *relres = s.last_rhob > 0 ? std::sqrt(std::max(s.last_rho, 0.0) / s.last_rhob) : 0.0;
  return flags_to_status(s.last_flags);
}

// ---------------------------------------------------------------------------------------
// Batches: many simulations advanced by one persistent kernel (batch_kernel)
// ---------------------------------------------------------------------------------------
struct dg_batch {
  int max_sims = 0;
  std::vector<dg_sim*> sims;
  int ngroups_req = 0;  // 0: automatic
  // launch configuration (dg_batch_set_tiles / dg_batch_set_blocks_per_sm / dg_batch_autotune):
  // per n the RHS and solve tiles (0: built-in) and a cap on resident blocks per SM (0: none)
  int tile_rhs[kMaxN + 1][2] = {};
  int tile_cg[kMaxN + 1][2] = {};
  int bps_cap = 0;
  std::vector<long long> tuned_key;  // the member classes the tuned configuration was found for
  char tuned_desc[512] = "";
  bool dirty = true;    // composition or plan changed: re-plan, re-upload, re-capture
  int stable = 0;       // launches since the last re-plan
  BatchSim* d_sims = nullptr;
  int* d_order = nullptr;
  BatchGroup* d_groups = nullptr;
  SyncState* d_sync = nullptr;
  int* d_error = nullptr;
  int cap_groups = 256;
  int grid = 0, ngroups = 0;
  size_t smem = 0;
  std::vector<int> order;
  std::vector<BatchGroup> groups;
  cudaGraphExec_t graph = nullptr;
  int graph_steps = 0;
  bool use_graph = true;
  char graph_error[256] = "";
  long long launches = 0;
  // pinned staging of the plan (uploaded asynchronously on the step's stream)
  BatchSim* h_sims = nullptr;
  int* h_order = nullptr;
  BatchGroup* h_groups = nullptr;
  cudaEvent_t ev_upload = nullptr;
  bool upload_pending = false;
};

namespace {

// Tiles of a simulation inside a batch: the batch's choice for its n, else the built-in ones
// (a small grid's blocks are few in a batch group, so its tiles are not split further as for a
// whole-GPU solve).
void batch_geoms(const dg_batch* b, const dg_grid* g, Geom* Gr, Geom* Gc) {
  int rty, rtx, cty, ctx;
  default_tiles(g->n, rty, rtx, cty, ctx);
  if (b && b->tile_rhs[g->n][0] > 0) {
    rty = b->tile_rhs[g->n][0];
    rtx = b->tile_rhs[g->n][1];
  }
  if (b && b->tile_cg[g->n][0] > 0) {
    cty = b->tile_cg[g->n][0];
    ctx = b->tile_cg[g->n][1];
  }
  *Gr = geom_of(g, rty, rtx);
  *Gc = geom_of(g, cty, ctx);
}

BatchSim make_batch_sim(const dg_batch* bt, dg_sim* s) {
  dg_grid* g = s->g;
  BatchSim b{};
  b.n = g->n;
  b.precision = s->precision == DG_FP64 ? 0 : (s->precision == DG_MIXED ? 1 : 2);
  b.precond = g->precond;
  batch_geoms(bt, g, &b.Gr, &b.Gc);
  b.ops_d = g->d_opsd;
  b.ops_f = g->d_opsf;
  b.ops_df = g->d_opsx;
  b.ops_k = g->d_opsk;
  b.precise_apply = g->precise_apply;
  b.keep_mean = g->bc;
  for (int i = 0; i < 2; ++i) b.omega[i] = s->omega[i];
  for (int i = 0; i < 3; ++i) {
    b.psi[i] = s->psi[i];
    b.apsi[i] = s->apsi[i];
    b.apsi_ok[i] = s->apsi_ok[i] ? 1 : 0;
  }
  for (int i = 0; i < 4; ++i) b.R[i] = s->R[i];
  b.oc = s->oc;
  b.p0 = s->p0;
  b.p1 = s->p1;
  b.p2 = s->p2;
  b.r1 = s->r1;
  b.r2 = s->r2;
  b.r3 = s->r3;
  b.rfree = s->rfree;
  b.step = s->step;
  b.limit = s->batch_limit;
  b.D = s->D;
  b.dt = s->dt;
  b.tol2 = s->tol * s->tol;
  b.floor2 = g->floor2;
  b.tol_in2 = s->tol_in * s->tol_in;
  b.maxit = s->maxit;
  b.max_sweeps = s->max_sweeps;
  b.fixed_iters = s->fixed_iters;
  b.sumW = g->Lx * g->Ly;
  b.r = s->ws.r;
  b.p0v = s->ws.p0;
  b.p1v = s->ws.p1;
  b.q = s->ws.q;
  b.part = s->ws.part;
  b.rf = s->ws.rf;
  b.fr = s->ws.fr;
  b.fe = s->ws.fe;
  b.fp0 = s->ws.fp0;
  b.fp1 = s->ws.fp1;
  b.fq = s->ws.fq;
  b.partf = s->ws.partf;
  b.status = s->ws.status;
  b.pc = pc_args(g, s->ws);
  b.pcf = pc_args_f(g, s->ws);
  return b;
}

// Dynamic shared memory one simulation needs in batch_kernel (RHS tile and solve share it).
size_t batch_smem_for(const dg_batch* b, const dg_sim* s) {
  const dg_grid* g = s->g;
  Geom Gr, Gc;
  batch_geoms(b, g, &Gr, &Gc);
  const int Lmax = std::max(g->Nx, g->Ny);
  size_t out = 0;
  dispatch_n(g->n, [&](auto nc) {
    constexpr int N = decltype(nc)::value;
    const size_t rhs = rhs_smem_values<double, N>(Gr.TY, Gr.TX) * sizeof(double);  // double or double-float
    const size_t sol = s->precision == DG_FP64 ? cg_smem_bytes<double, N>(Gc.TY, Gc.TX, Lmax, g->precond, pow2_grid(g))
                                               : mixed_smem_bytes<N>(Gc.TY, Gc.TX, Lmax, g->precond, pow2_grid(g));
    out = batch_ops_bytes<N>() + std::max(rhs, sol);
    return DG_OK;
  });
  return out;
}

// Splits the simulations into groups of balanced work (longest processing time first; work
// ~ dof) and the co-resident blocks among the groups in proportion to their work.
int batch_plan(dg_batch* b, int dev_sms, cudaStream_t st) {
  const int ns = (int)b->sims.size();
  size_t smem = 0;
  for (dg_sim* s : b->sims) smem = std::max(smem, batch_smem_for(b, s));
  int optin = 0;
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  if (smem > (size_t)optin) return fail(DG_ERR_ARG, "batch needs %zu B of shared memory per block (max %d)", smem, optin);
  int per_sm = 0;
  if (int rc = batch_kernel_occupancy(smem, &per_sm)) return rc;
  if (per_sm < 1) return fail(DG_ERR_CUDA, "batch kernel does not fit on an SM");
  if (b->bps_cap > 0) per_sm = std::min(per_sm, b->bps_cap);
  int grid = per_sm * dev_sms;
  for (dg_sim* s : b->sims) grid = std::min(grid, s->ws.grid_cap);
  int G = b->ngroups_req > 0 ? b->ngroups_req : std::min(ns, 8);
  G = std::max(1, std::min({G, ns, grid, b->cap_groups}));
  std::vector<int> idx(ns);
  for (int i = 0; i < ns; ++i) idx[i] = i;
  auto work = [&](int i) { return (double)ndof_of(b->sims[i]->g); };
  std::sort(idx.begin(), idx.end(), [&](int a, int c) { return work(a) > work(c); });
  std::vector<double> gw(G, 0.0);
  std::vector<std::vector<int>> members(G);
  for (int i : idx) {
    const int k = int(std::min_element(gw.begin(), gw.end()) - gw.begin());
    gw[k] += work(i);
    members[k].push_back(i);
  }
  double total = 0.0;
  for (double w : gw) total += w;
  std::vector<int> nb(G, 1);
  int left = grid - G;
  for (int k = 0; k < G && left > 0; ++k) {
    const int extra = std::min(left, int(std::floor((grid - G) * gw[k] / total)));
    nb[k] += extra;
    left -= extra;
  }
  for (int k = 0; left > 0; k = (k + 1) % G, --left) nb[k] += 1;
  b->order.clear();
  b->groups.assign(G, BatchGroup{});
  int fb = 0;
  for (int k = 0; k < G; ++k) {
    b->groups[k].first_block = fb;
    b->groups[k].nblocks = nb[k];
    b->groups[k].first = (int)b->order.size();
    b->groups[k].count = (int)members[k].size();
    b->groups[k].sync = b->d_sync + k;
    for (int i : members[k]) b->order.push_back(i);
    fb += nb[k];
  }
  // the staging buffers are rewritten only after the previous upload has executed
  if (b->upload_pending) CUDA_TRY(cudaEventSynchronize(b->ev_upload));
  for (int i = 0; i < ns; ++i) b->h_sims[i] = make_batch_sim(b, b->sims[i]);
  std::copy(b->order.begin(), b->order.end(), b->h_order);
  std::copy(b->groups.begin(), b->groups.end(), b->h_groups);
  CUDA_TRY(cudaMemcpyAsync(b->d_sims, b->h_sims, ns * sizeof(BatchSim), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b->d_order, b->h_order, ns * sizeof(int), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaMemcpyAsync(b->d_groups, b->h_groups, G * sizeof(BatchGroup), cudaMemcpyHostToDevice, st));
  CUDA_TRY(cudaEventRecord(b->ev_upload, st));
  b->upload_pending = true;
  b->grid = grid;
  b->ngroups = G;
  b->smem = smem;
  if (b->graph) {
    cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
  }
  b->dirty = false;
  b->stable = 0;
  return DG_OK;
}

int batch_enqueue(dg_batch* b, int nsteps, cudaStream_t st) {
  CUDA_TRY(cudaMemsetAsync(b->d_sync, 0, b->ngroups * sizeof(SyncState), st));
  BatchArgs A{b->d_sims, b->d_order, b->d_groups, b->ngroups, nsteps, b->d_error};
  if (int rc = batch_kernel_launch(A, b->grid, b->smem, st)) return rc;
  return DG_OK;
}

// Host mirror of the rotations the kernel applies to every simulation per step.
void batch_advance_host(dg_batch* b, int nsteps) {
  for (dg_sim* s : b->sims)
    for (int k = 0; k < nsteps; ++k) {
      if (s->batch_limit > 0 && s->step >= s->batch_limit) break;
      s->oc ^= 1;
      const int p0 = s->p0, p1 = s->p1, p2 = s->p2;
      s->apsi_ok[p2] = s->fixed_iters == 0;
      s->p0 = p2;
      s->p1 = p0;
      s->p2 = p1;
      rotate_history(s);
      s->step += 1;
    }
}

}  // namespace

extern "C" {

int dg_batch_create(dg_batch** bp, int max_sims) {
  if (!bp || max_sims < 1) return fail(DG_ERR_ARG, "bad arguments");
  *bp = nullptr;
  dg_batch* b = new (std::nothrow) dg_batch();
  if (!b) return fail(DG_ERR_NOMEM, "host allocation failed");
  b->max_sims = max_sims;
  auto alloc = [&]() -> int {
    CUDA_TRY(cudaMalloc(&b->d_sims, max_sims * sizeof(BatchSim)));
    CUDA_TRY(cudaMalloc(&b->d_order, max_sims * sizeof(int)));
    CUDA_TRY(cudaMalloc(&b->d_groups, b->cap_groups * sizeof(BatchGroup)));
    CUDA_TRY(cudaMalloc(&b->d_sync, b->cap_groups * sizeof(SyncState)));
    CUDA_TRY(cudaMalloc(&b->d_error, sizeof(int)));
    CUDA_TRY(cudaMemset(b->d_error, 0, sizeof(int)));
    CUDA_TRY(cudaMallocHost(&b->h_sims, max_sims * sizeof(BatchSim)));
    CUDA_TRY(cudaMallocHost(&b->h_order, max_sims * sizeof(int)));
    CUDA_TRY(cudaMallocHost(&b->h_groups, b->cap_groups * sizeof(BatchGroup)));
    CUDA_TRY(cudaEventCreateWithFlags(&b->ev_upload, cudaEventDisableTiming));
    return DG_OK;
  };
  if (int rc = alloc()) {
    dg_batch_destroy(b);
    return rc;
  }
  *bp = b;
  return DG_OK;
}

int dg_batch_destroy(dg_batch* b) {
  if (!b) return DG_OK;
  if (b->graph) cudaGraphExecDestroy(b->graph);
  cudaFree(b->d_sims);
  cudaFree(b->d_order);
  cudaFree(b->d_groups);
  cudaFree(b->d_sync);
  cudaFree(b->d_error);
  if (b->h_sims) cudaFreeHost(b->h_sims);
  if (b->h_order) cudaFreeHost(b->h_order);
  if (b->h_groups) cudaFreeHost(b->h_groups);
  if (b->ev_upload) cudaEventDestroy(b->ev_upload);
  delete b;
  return DG_OK;
}

int dg_batch_admit(dg_batch* b, dg_sim* s, void* stream) {
  if (!b || !s) return fail(DG_ERR_ARG, "NULL argument");
  if ((int)b->sims.size() >= b->max_sims) return fail(DG_ERR_NOMEM, "batch is full (%d simulations)", b->max_sims);
  for (dg_sim* t : b->sims)
    if (t == s) return fail(DG_ERR_ARG, "simulation already in the batch");
  if (s->K != 3) return fail(DG_ERR_ARG, "batched steps are AB3 (the simulation uses K = %d)", s->K);
  if (s->precision == DG_FP64_PC32) return fail(DG_ERR_ARG, "batched simulations use DG_FP64, DG_MIXED or DG_MIXED64");
  if (s->parts != 0) return fail(DG_ERR_ARG, "batched steps use the bracket of Eq. J");
  if (s->step < 2)
    if (int rc = dg_step(s, int(2 - s->step), stream)) return rc;  // RK4 start-up steps on their own
  b->sims.push_back(s);
  b->dirty = true;
  return DG_OK;
}

int dg_batch_retire(dg_batch* b, dg_sim* s) {
  if (!b || !s) return fail(DG_ERR_ARG, "NULL argument");
  for (size_t i = 0; i < b->sims.size(); ++i)
    if (b->sims[i] == s) {
      b->sims.erase(b->sims.begin() + i);
      b->dirty = true;
      return DG_OK;
    }
  return fail(DG_ERR_ARG, "simulation not in the batch");
}

int dg_batch_size(const dg_batch* b) { return b ? (int)b->sims.size() : 0; }

int dg_batch_set_limit(dg_batch* b, dg_sim* s, long long last_step) {
  if (!b || !s || last_step < 0) return fail(DG_ERR_ARG, "bad arguments");
  s->batch_limit = last_step;
  for (dg_sim* t : b->sims)
    if (t == s) b->dirty = true;  // the limit travels with the plan's descriptors
  return DG_OK;
}

int dg_batch_set_groups(dg_batch* b, int ngroups) {
  if (!b || ngroups < 0) return fail(DG_ERR_ARG, "bad arguments");
  b->ngroups_req = ngroups;
  b->dirty = true;
  return DG_OK;
}

int dg_batch_set_tiles(dg_batch* b, int n, int rhs_ty, int rhs_tx, int cg_ty, int cg_tx) {
  if (!b || n < 1 || n > kMaxN) return fail(DG_ERR_ARG, "bad arguments");
  const int t[4] = {rhs_ty, rhs_tx, cg_ty, cg_tx};
  for (int v : t)
    if (v < 0 || v > 64) return fail(DG_ERR_ARG, "tile sides must be 0..64 cells");
  if ((rhs_ty == 0) != (rhs_tx == 0) || (cg_ty == 0) != (cg_tx == 0))
    return fail(DG_ERR_ARG, "give both sides of a tile, or 0 for both (built-in)");
  b->tile_rhs[n][0] = rhs_ty;
  b->tile_rhs[n][1] = rhs_tx;
  b->tile_cg[n][0] = cg_ty;
  b->tile_cg[n][1] = cg_tx;
  b->dirty = true;
  return DG_OK;
}

int dg_batch_set_blocks_per_sm(dg_batch* b, int cap) {
  if (!b || cap < 0) return fail(DG_ERR_ARG, "bad arguments");
  b->bps_cap = cap;
  b->dirty = true;
  return DG_OK;
}

int dg_batch_get_config(const dg_batch* b, char* buf, int len) {
  if (!b || !buf || len < 1) return fail(DG_ERR_ARG, "bad arguments");
  int off = snprintf(buf, len, "groups=%d blocks_per_sm=%d grid=%d", b->ngroups, b->bps_cap, b->grid);
  for (int n = 1; n <= kMaxN && off < len; ++n) {
    bool present = false;
    for (const dg_sim* s : b->sims) present = present || s->g->n == n;
    if (!present) continue;
    int rty, rtx, cty, ctx;
    default_tiles(n, rty, rtx, cty, ctx);
    if (b->tile_rhs[n][0] > 0) {
      rty = b->tile_rhs[n][0];
      rtx = b->tile_rhs[n][1];
    }
    if (b->tile_cg[n][0] > 0) {
      cty = b->tile_cg[n][0];
      ctx = b->tile_cg[n][1];
    }
    off += snprintf(buf + off, len - off, " n%d:rhs=%dx%d,cg=%dx%d", n, rty, rtx, cty, ctx);
  }
  return DG_OK;
}

int dg_batch_step(dg_batch* b, int nsteps, void* stream);

int dg_batch_autotune(dg_batch* b, int trial_steps, void* stream) {
  if (!b || trial_steps < 1) return fail(DG_ERR_ARG, "bad arguments");
  if (b->sims.empty()) return DG_OK;
  cudaStream_t st = as_stream(stream);
  // the member classes: a configuration found for the same classes is reused
  std::vector<long long> key;
  for (const dg_sim* s : b->sims)
    key.push_back(((long long)s->g->Nx * 100000 + s->g->Ny) * 100 + s->g->n * 10 + s->precision);
  std::sort(key.begin(), key.end());
  if (key == b->tuned_key) return DG_OK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  const bool use_graph = b->use_graph;
  b->use_graph = false;  // every trial is a fresh plan launched directly
  int rc = DG_OK;
  auto trial = [&](float* ms) -> int {
    b->dirty = true;
    if (int r = dg_batch_step(b, 1, stream)) return r;  // the new plan's first launch (uploads)
    CUDA_TRY(cudaEventRecord(e0, st));
    if (int r = dg_batch_step(b, trial_steps, stream)) return r;
    CUDA_TRY(cudaEventRecord(e1, st));
    CUDA_TRY(cudaEventSynchronize(e1));
    CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
    *ms /= float(trial_steps);
    return DG_OK;
  };
  float best = 0.f;
  rc = trial(&best);
  const int ns = (int)b->sims.size();
  // the classes of n, the largest total dof first
  std::vector<std::pair<double, int>> by_n;
  for (int n = 1; n <= kMaxN; ++n) {
    double w = 0.0;
    for (const dg_sim* s : b->sims)
      if (s->g->n == n) w += (double)ndof_of(s->g);
    if (w > 0.0) by_n.push_back({w, n});
  }
  std::sort(by_n.rbegin(), by_n.rend());
  static const int kRhsTiles[][2] = {{2, 4}, {4, 4}, {4, 8}, {8, 8}, {8, 16}, {16, 16}};
  static const int kCgTiles[][2] = {{4, 8}, {8, 8}, {8, 16}, {16, 16}};
  // Coordinate descent, two rounds (a tile's shared memory sets how many blocks of the whole
  // batch fit on an SM, so one choice changes what the others are worth): the number of block
  // groups; per n the RHS tile, then the solve tile; a cap on blocks per SM.  A candidate whose
  // shared memory does not fit is skipped.
  for (int round = 0; round < 2 && !rc; ++round) {
    int bestG = b->ngroups_req;
    for (int G : {1, 2, 4, 8, 16, 32}) {
      if (G > ns || G == b->ngroups) continue;
      b->ngroups_req = G;
      float ms = 0.f;
      if ((rc = trial(&ms))) break;
      if (ms < best) {
        best = ms;
        bestG = G;
      }
    }
    b->ngroups_req = bestG;
    for (auto& wn : by_n) {
      const int n = wn.second;
      for (int which = 0; which < 2 && !rc; ++which) {
        int(*tile)[2] = which == 0 ? b->tile_rhs : b->tile_cg;
        const int(*cand)[2] = which == 0 ? kRhsTiles : kCgTiles;
        const int ncand = which == 0 ? 6 : 4;
        int keep[2] = {tile[n][0], tile[n][1]};
        for (int c = 0; c < ncand; ++c) {
          if (cand[c][0] == keep[0] && cand[c][1] == keep[1]) continue;
          tile[n][0] = cand[c][0];
          tile[n][1] = cand[c][1];
          float ms = 0.f;
          const int r = trial(&ms);
          if (r == DG_ERR_ARG) continue;  // this tile's shared memory does not fit
          if ((rc = r)) break;
          if (ms < best) {
            best = ms;
            keep[0] = cand[c][0];
            keep[1] = cand[c][1];
          }
        }
        tile[n][0] = keep[0];
        tile[n][1] = keep[1];
      }
    }
    if (!rc) {
      int keep = b->bps_cap;
      for (int cap : {0, 1, 2, 3}) {
        if (cap == keep) continue;
        b->bps_cap = cap;
        float ms = 0.f;
        if ((rc = trial(&ms))) break;
        if (ms < best) {
          best = ms;
          keep = cap;
        }
      }
      b->bps_cap = keep;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->use_graph = use_graph;
  b->dirty = true;
  if (rc) return rc;
  b->tuned_key = key;
  return DG_OK;
}

int dg_batch_step(dg_batch* b, int nsteps, void* stream) {
  if (!b || nsteps < 0) return fail(DG_ERR_ARG, "bad arguments");
  if (b->sims.empty() || nsteps == 0) return DG_OK;
  cudaStream_t st = as_stream(stream);
  int dev = 0, sms = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (b->dirty)
    if (int rc = batch_plan(b, sms, st)) return rc;
  // a CUDA graph once the plan has served two launches unchanged (a batch whose members
  // change at every launch, as under continuous batching, launches directly)
  if (b->use_graph && b->stable >= 2 && (!b->graph || b->graph_steps != nsteps)) {
    if (b->graph) {
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
    cudaStream_t cs;
    CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int rc_enq = (e == cudaSuccess) ? batch_enqueue(b, nsteps, cs) : DG_ERR_CUDA;
    const cudaError_t e_end = cudaStreamEndCapture(cs, &graph);
    if (e == cudaSuccess) e = e_end;
    if (e == cudaSuccess && rc_enq == DG_OK && graph) e = cudaGraphInstantiate(&b->graph, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaGetLastError();
    if (e != cudaSuccess || rc_enq != DG_OK || !b->graph) {
      snprintf(b->graph_error, sizeof(b->graph_error), "%s", e != cudaSuccess ? cudaGetErrorString(e) : g_err);
      b->graph = nullptr;
      b->use_graph = false;  // fall back to direct cooperative launches
    } else {
      b->graph_steps = nsteps;
    }
  }
  if (b->graph) {
    CUDA_TRY(cudaGraphLaunch(b->graph, st));
  } else if (int rc = batch_enqueue(b, nsteps, st)) {
    return rc;
  }
  b->launches += 1;
  b->stable += 1;
  batch_advance_host(b, nsteps);
  return DG_OK;
}

int dg_batch_status(dg_batch* b, int* uses_graph, int* ngroups, long long* launches, void* stream) {
  if (!b) return fail(DG_ERR_ARG, "NULL argument");
  int err = 0;
  CUDA_TRY(cudaMemcpyAsync(&err, b->d_error, sizeof(int), cudaMemcpyDeviceToHost, as_stream(stream)));
  CUDA_TRY(cudaStreamSynchronize(as_stream(stream)));
  if (uses_graph) *uses_graph = b->graph ? 1 : 0;
  if (!b->graph && b->graph_error[0]) snprintf(g_err, sizeof(g_err), "graph capture unavailable: %s", b->graph_error);
  if (ngroups) *ngroups = b->ngroups;
  if (launches) *launches = b->launches;
  if (err) return fail(DG_ERR_TIMEOUT, "a device-side wait of the batched kernel hit its cap");
  for (dg_sim* s : b->sims) {
    SolveStatus ss;
    if (int rc = read_status(s->ws, &ss, as_stream(stream))) return rc;
    if (ss.flags) return flags_to_status(ss.flags);
  }
  return DG_OK;
}

}  // extern "C"
