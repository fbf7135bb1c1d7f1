// The hot-path kernels, templated on the arithmetic type T (double or float) and the
// number of nodes per cell and dimension N (1..5).
//
//   rhs_kernel       bracket J(psi, omega) (Eq. J) + viscous term + multistep update, fused
//   apply_kernel     the LDG operator A or Delta_h on a field
//   cg_kernel        persistent cooperative conjugate-gradient Poisson solve (Sec. 6)
//   mixed_cg_kernel  float64 residual / float32 inner CG iterative refinement
//   invariants_*     V, E, Omega by quadrature (Eq. quantities, Eq. def_norm)
#pragma once

#include <type_traits>

#include "dg_device.cuh"
#include "dg_df.cuh"

namespace dgk {

constexpr int kThreads = 256;
// Threads of a standalone RHS block: its tile's staging (up to about 190 KB at n = 5) leaves
// room for one or two blocks per SM, so the block itself must carry the SM's warps (measured on
// the 1024^2, n = 5 step: 6.56 / 5.47 / 5.07 ms per RHS with 256 / 512 / 1024 threads; on
// 512^2, n = 4: 1.01 / 0.88 / 1.12 ms).
template <int N>
__host__ __device__ constexpr int rhs_threads() {
  return N == 5 ? 1024 : 512;
}

// Copies an operator table (a kernel parameter or a global array) to shared memory: the
// solves index it with per-thread node numbers, which shared memory serves without the
// serialisation of divergent constant-bank reads.
template <class Tab>
__device__ __forceinline__ const Tab& stage_table(const Tab& src, unsigned char* dst) {
  static_assert(sizeof(Tab) % 4 == 0, "table size");
  const unsigned int* s = reinterpret_cast<const unsigned int*>(&src);
  unsigned int* d = reinterpret_cast<unsigned int*>(dst);
  for (int i = threadIdx.x; i < int(sizeof(Tab) / 4); i += blockDim.x) d[i] = s[i];
  __syncthreads();
  return *reinterpret_cast<const Tab*>(dst);
}

template <class Tab>
__host__ __device__ constexpr size_t table_bytes() {
  return (sizeof(Tab) + 15) & ~size_t(15);
}


__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ df mul_rn(df a, df b) { return a * b; }
__device__ __forceinline__ df sub_rn(df a, df b) { return a - b; }

// Storage type of the right-hand-side history for an RHS evaluated in T: float64 for the
// float64 and the double-float bracket (a double-float value converts to float64 exactly).
template <typename T>
struct HistType {
  using type = double;
};
template <>
struct HistType<float> {
  using type = float;
};
template <typename T>
using hist_t = typename HistType<T>::type;

// a*b - c*d with both products rounded separately (never contracted into an FMA), so that
// the bracket's antisymmetry J(f, g) = -J(g, f) and J(f, f) = 0 hold bitwise.
template <typename T>
__device__ __forceinline__ T prod_diff(T a, T b, T c, T d) {
  return sub_rn(mul_rn(a, b), mul_rn(c, d));
}

// =========================================================================================
// Right-hand side: R = -J(psi, omega) + D Delta_h omega and the update
//   omega_out = omega_base + dt (c_new R + sum_m c_hist[m] hist[m])
// (AB3: c = 23/12, -16/12, 5/12; the RK4 start-up stages use other coefficients).
// One thread block per tile of TY x TX cells; the tile and a one-cell halo ring (corners
// included: the second derivatives of J+x and Jx+ reach the diagonal neighbours) are staged
// in shared memory, all intermediate products stay there.
// =========================================================================================
template <typename T>
struct RhsArgs {
  const double* psi;        // stream function; times sqrt(W) if psi_scaled
  const double* omega_in;   // vorticity at which R is evaluated (halo reads)
  const double* omega_base; // omega^k of the update (own nodes only; may alias omega_out)
  double* omega_out;        // updated vorticity, or J in bracket-only mode
  hist_t<T>* R_out;         // fresh R (may alias one hist buffer); may be null
  const hist_t<T>* hist[3];
  double c_new;
  double c_hist[3];
  int nhist;
  double dt;
  double visc;
  int psi_scaled;
  int bracket_only;
  int parts;                // bit 0: J++, bit 1: J+x, bit 2: Jx+ (0 = all three, J of Eq. J)
};

template <typename T, int N>
__host__ __device__ constexpr size_t rhs_smem_values(int TY, int TX) {
  return (size_t)(TY + 2) * (TX + 2) * (7 * (N * N + 1) + 12 * N);
}

// One tile of the right-hand side (smem: rhs_smem_values<T, N>(G.TY, G.TX) values of T).
template <typename T, int N>
__device__ __forceinline__ void rhs_tile(const Ops2D<T, N>& C, const Geom& G, const RhsArgs<T>& A, int tile,
                                         unsigned char* smem_raw) {
  constexpr int NN = N * N;
  constexpr int CS = NN + 1;  // padded cell stride in shared memory
  T* sm = reinterpret_cast<T*>(smem_raw);
  const TileBox B = make_box(G, tile);
  const int boxc = (G.TY + 2) * (G.TX + 2);
  T* sPsi = sm;
  T* sOm = sPsi + boxc * CS;
  T* sFx = sOm + boxc * CS;  // f_x, later h2 = f_x g - f g_x   (cells with rx in [0,TXe))
  T* sGx = sFx + boxc * CS;
  T* sFy = sGx + boxc * CS;  // f_y, later h1 = f g_y - f_y g   (cells with ry in [0,TYe))
  T* sGy = sFy + boxc * CS;
  T* sJ = sGy + boxc * CS;   // J++ on the tile
  T* t0 = sJ + boxc * CS;
  T *tPxR = t0, *tPxL = t0 + boxc * N, *tPyR = t0 + 2 * boxc * N, *tPyL = t0 + 3 * boxc * N;
  T *tOxR = t0 + 4 * boxc * N, *tOxL = t0 + 5 * boxc * N, *tOyR = t0 + 6 * boxc * N, *tOyL = t0 + 7 * boxc * N;
  T *tLxR = t0 + 8 * boxc * N, *tLxL = t0 + 9 * boxc * N, *tLyR = t0 + 10 * boxc * N, *tLyL = t0 + 11 * boxc * N;
  const int BW = B.BW;

  // S0: stage psi and omega on the tile with its full halo ring.
  stage_box<T, N>(G, B, sPsi, true, [&](size_t g, int k, bool) {
    const double v = A.psi[g];
    return A.psi_scaled ? T(v) * C.isw[k] : T(v);
  });
  stage_box<T, N>(G, B, sOm, true, [&](size_t g, int, bool) { return T(A.omega_in[g]); });
  __syncthreads();

  // S1: face traces for the first derivatives (every staged cell) and the viscous term.
  line_traces<T, N>(B, sPsi, sPsi, C.dx, C.dy, tPxR, tPxL, tPyR, tPyL, true);
  line_traces<T, N>(B, sOm, sOm, C.dx, C.dy, tOxR, tOxL, tOyR, tOyL, true);
  if (A.visc != 0.0) line_traces<T, N>(B, sOm, sOm, C.lx, C.ly, tLxR, tLxL, tLyR, tLyL, false);
  __syncthreads();
  if (G.bc) {  // Dirichlet: f^ = 0 on the boundary faces of the derivatives; LDG first cells
    dirichlet_ghost_traces<T, N>(G, B, tPxR, tPxL, tPyR, tPyL, true);
    dirichlet_ghost_traces<T, N>(G, B, tOxR, tOxL, tOyR, tOyL, true);
    if (A.visc != 0.0) dirichlet_first_traces<T, N>(B, sOm, sOm, C.lx, C.ly, tLxL, tLyL);
    __syncthreads();
  }

  // S2: f_x, g_x on rows [-1, TYe] x cols [0, TXe); f_y, g_y on rows [0, TYe) x cols [-1, TXe].
  {
    const int n1 = (B.TYe + 2) * B.TXe * NN;
    const int n2 = B.TYe * (B.TXe + 2) * NN;
    for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
      if (i < n1) {
        const int c = i / NN, k = i - (i / NN) * NN;
        const int ry = quot(c, B.mTXe) - 1, rx = c - (ry + 1) * B.TXe;
        const int lc = (ry + 1) * BW + rx + 1;
        const int a = k / N, b = k - (k / N) * N;
        sFx[lc * CS + k] = op_x_at<T, N>(sPsi, tPxR, tPxL, C.dx, lc, a, b);
        sGx[lc * CS + k] = op_x_at<T, N>(sOm, tOxR, tOxL, C.dx, lc, a, b);
      } else {
        const int ii = i - n1;
        const int c = ii / NN, k = ii - (ii / NN) * NN;
        const int w = B.TXe + 2;
        const int ry = c / w, rx = c - (c / w) * w - 1;
        const int lc = (ry + 1) * BW + rx + 1;
        const int a = k / N, b = k - (k / N) * N;
        sFy[lc * CS + k] = op_y_at<T, N>(sPsi, tPyR, tPyL, C.dy, lc, BW, a, b);
        sGy[lc * CS + k] = op_y_at<T, N>(sOm, tOyR, tOyL, C.dy, lc, BW, a, b);
      }
    }
  }
  __syncthreads();

  // Which parts enter (Eq. J): J = s (c0 J++ + J+x + Jx+) with J+x = D_x(f g_y) - D_y(f g_x),
  // Jx+ = D_y(f_x g) - D_x(f_y g); as h1 = a1 f g_y - b1 f_y g, h2 = a2 f_x g - b2 f g_x.
  const int parts = A.parts ? A.parts : 7;
  const bool use_pp = parts & 1, use_px = parts & 2, use_xp = parts & 4;
  const int nparts = int(use_pp) + int(use_px) + int(use_xp);
  // S3a: J++ = f_x g_y - f_y g_x on the tile.
  const int nin = B.TYe * B.TXe * NN;
  for (int i = threadIdx.x; i < nin; i += blockDim.x) {
    const int c = i / NN, k = i - (i / NN) * NN;
    const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
    const int o = ((ry + 1) * BW + rx + 1) * CS + k;
    sJ[o] = prod_diff(sFx[o], sGy[o], sFy[o], sGx[o]);
  }
  __syncthreads();

  // S3b: h1 = f g_y - f_y g (in place of f_y), h2 = f_x g - f g_x (in place of f_x).
  {
    const int n1 = B.TYe * (B.TXe + 2) * NN;
    const int n2 = (B.TYe + 2) * B.TXe * NN;
    for (int i = threadIdx.x; i < n1 + n2; i += blockDim.x) {
      if (i < n1) {
        const int c = i / NN, k = i - (i / NN) * NN;
        const int w = B.TXe + 2;
        const int ry = c / w, rx = c - (c / w) * w - 1;
        const int o = ((ry + 1) * BW + rx + 1) * CS + k;
        if (nparts == 3)
          sFy[o] = prod_diff(sPsi[o], sGy[o], sFy[o], sOm[o]);
        else
          sFy[o] = (use_px ? mul_rn(sPsi[o], sGy[o]) : T(0)) - (use_xp ? mul_rn(sFy[o], sOm[o]) : T(0));
      } else {
        const int ii = i - n1;
        const int c = ii / NN, k = ii - (ii / NN) * NN;
        const int ry = quot(c, B.mTXe) - 1, rx = c - (ry + 1) * B.TXe;
        const int o = ((ry + 1) * BW + rx + 1) * CS + k;
        if (nparts == 3)
          sFx[o] = prod_diff(sFx[o], sOm[o], sPsi[o], sGx[o]);
        else
          sFx[o] = (use_xp ? mul_rn(sFx[o], sOm[o]) : T(0)) - (use_px ? mul_rn(sPsi[o], sGx[o]) : T(0));
      }
    }
  }
  __syncthreads();

  // S4: traces of h1 along x and of h2 along y (reusing the psi trace arrays).
  line_traces<T, N>(B, sFy, sFx, C.dx, C.dy, tPxR, tPxL, tPyR, tPyL, false);
  __syncthreads();
  if (G.bc) {
    dirichlet_ghost_traces<T, N>(G, B, tPxR, tPxL, tPyR, tPyL, false);
    __syncthreads();
  }

  // S5: J = (J++ + D_x h1 + D_y h2) / 3 = (J++ + J+x + Jx+) / 3, the viscous term and the update.
  const T third = nparts == 3 ? T(1.0 / 3.0) : T(1);
  for (int i = threadIdx.x; i < nin; i += blockDim.x) {
    const int c = i / NN, k = i - (i / NN) * NN;
    const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
    const int lc = (ry + 1) * BW + rx + 1;
    const int a = k / N, b = k - (k / N) * N;
    const T dxh1 = op_x_at<T, N>(sFy, tPxR, tPxL, C.dx, lc, a, b);
    const T dyh2 = op_y_at<T, N>(sFx, tPyR, tPyL, C.dy, lc, BW, a, b);
    const T J = (((use_pp ? sJ[lc * CS + k] : T(0)) + dxh1) + dyh2) * third;
    const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
    if (A.bracket_only) {
      A.omega_out[g] = double(J);
      continue;
    }
    T R = -J;
    if (A.visc != 0.0) {
      const bool fx = G.bc && B.tx0 + rx == 0, fy = G.bc && B.ty0 + ry == 0;
      const T lap = op_x_at<T, N>(sOm, tLxR, tLxL, C.lx, lc, a, b, fx) +
                    op_y_at<T, N>(sOm, tLyR, tLyL, C.ly, lc, BW, a, b, fy);
      R = fma(-T(A.visc), lap, R);  // + D Delta_h omega, since -Delta_h = lx + ly
    }
    double incr = A.c_new * double(R);
    for (int m = 0; m < A.nhist; ++m) incr = fma(A.c_hist[m], double(A.hist[m][g]), incr);
    if (A.R_out) A.R_out[g] = hist_t<T>(R);
    A.omega_out[g] = fma(A.dt, incr, A.omega_base[g]);
  }
  __syncthreads();
}

template <typename T, int N>
__global__ void __launch_bounds__(rhs_threads<N>()) rhs_kernel(const __grid_constant__ Ops2D<T, N> C, const Geom G,
                                                      const __grid_constant__ RhsArgs<T> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  rhs_tile<T, N>(stage_table(C, smem_raw), G, A, blockIdx.x, smem_raw + table_bytes<Ops2D<T, N>>());
}

// =========================================================================================
// Operator application: mode 0  y = A x = W^1/2 (W^-1/2 A W^-1/2) W^1/2 x,
//                       mode 1  y = Delta_h x = -(lx + ly) x.
// =========================================================================================
template <typename T, int N>
__host__ __device__ constexpr size_t apply_smem_values(int TY, int TX) {
  return (size_t)(TY + 2) * (TX + 2) * (N * N + 1 + 4 * N);
}

template <typename T, int N>
__global__ void __launch_bounds__(kThreads) apply_kernel(const __grid_constant__ Ops2D<T, N> Cp, const Geom G,
                                                        const double* __restrict__ x, double* __restrict__ y,
                                                        int mode) {
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Ops2D<T, N>& C = stage_table(Cp, smem_raw);
  T* sU = reinterpret_cast<T*>(smem_raw + table_bytes<Ops2D<T, N>>());
  const int boxc = (G.TY + 2) * (G.TX + 2);
  T *tXR = sU + boxc * (NN + 1), *tXL = tXR + boxc * N, *tYR = tXL + boxc * N, *tYL = tYR + boxc * N;
  const TileBox B = make_box(G, blockIdx.x);
  const Op1D<T, N>& ox = mode == 0 ? C.kx : C.lx;
  const Op1D<T, N>& oy = mode == 0 ? C.ky : C.ly;
  stage_box<T, N>(G, B, sU, false, [&](size_t g, int k, bool) {
    return mode == 0 ? T(x[g]) * C.sw[k] : T(x[g]);
  });
  __syncthreads();
  line_traces<T, N>(B, sU, sU, ox, oy, tXR, tXL, tYR, tYL, false);
  __syncthreads();
  if (G.bc) {
    dirichlet_first_traces<T, N>(B, sU, sU, ox, oy, tXL, tYL);
    __syncthreads();
  }
  const int nin = B.TYe * B.TXe * NN;
  for (int i = threadIdx.x; i < nin; i += blockDim.x) {
    const int c = i / NN, k = i - (i / NN) * NN;
    const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
    const int lc = (ry + 1) * B.BW + rx + 1;
    const int a = k / N, b = k - (k / N) * N;
    const bool fx = G.bc && B.tx0 + rx == 0, fy = G.bc && B.ty0 + ry == 0;
    const T q = op_x_at<T, N>(sU, tXR, tXL, ox, lc, a, b, fx) + op_y_at<T, N>(sU, tYR, tYL, oy, lc, B.BW, a, b, fy);
    const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
    y[g] = mode == 0 ? double(q * C.sw[k]) : -double(q);
  }
}

// =========================================================================================
// Persistent conjugate-gradient solve of  Ahat y = b,  Ahat = W^-1/2 A W^-1/2  (plain CG on
// the symmetrically scaled system = CG on A psi = W omega preconditioned by W^-1, Sec. 6).
// Phases are separated by a capped grid barrier; dot products are block partials summed by
// every block in a fixed order (bit-identical scalars in all blocks, so every block takes the
// same branch).  Partial buffers alternate between two halves so that a block writing the
// next partial never races a slower block still reading the previous ones.
// =========================================================================================
constexpr int kRefineHistory = 48;  // sweeps recorded in SolveStatus

struct SolveStatus {
  long long total_iters;
  int last_iters;
  int max_iters;
  int flags;        // OR of all solves' flags
  int last_flags;
  int nsolves;
  int last_sweeps;  // refinement sweeps of the last mixed solve
  double last_rho;  // r.r of the last solve (scaled space)
  double last_rhob; // b.b
  // convergence history of the last mixed solve: r.r / b.b of the float64 residual before
  // sweep j (j = 0: of the initial guess) and the inner iterations of sweep j
  int hist_len;
  double hist_rr[kRefineHistory];
  int hist_it[kRefineHistory];
};

template <typename T>
struct CgVectors {
  T* y;      // solution (scaled space)
  T* r;      // residual
  T* p0;     // search directions (double-buffered: a phase reads one, writes the other)
  T* p1;
  T* q;      // Ahat p
};

template <typename T>
struct RhsSource {
  const double* omega;
  const T* rhs;
  T wbar;
};

template <typename T, int N>
__device__ __forceinline__ T rhs_at(const Ops2D<T, N>& C, const RhsSource<T>& B, size_t g, int k) {
  return B.rhs ? B.rhs[g] : C.sw[k] * (T(B.omega[g]) - B.wbar);
}

// Restarts from the true residual allowed after the recursive one has met the tolerance.
constexpr int kMaxRestarts = 20;

// ---- the two-level preconditioner --------------------------------------------------------
// In the scaled space (r~ = W^-1/2 r) the preconditioner M^-1 = B + P A_c^+ P^T of the
// unscaled system reads  z~ = Bt r~ + sqrt(W) (A_c^+ rc),  rc = sum over a cell's nodes of
// sqrt(W) r~  (= P^T r),  Bt = diag(sqrt W) A_cc^-1 diag(sqrt W)  (one n^2 x n^2 matrix for
// every cell), A_c = P^T A P the Galerkin coarse operator on the cells, diagonalised by the
// 2D DFT with eigenvalues ax[kx] + ay[ky] (constant mode dropped).
//
// The spectral preconditioner is M^-1 = Ahat^+ itself.  On the uniform periodic grid
// Ahat = I (x) Kx + Ky (x) I is block-circulant along both cell indices, so the DFT over cells
// turns each 1D operator into one n x n Hermitian matrix per wave number,
// Kx(kx) = M + e^{i th} a r^T + e^{-i th} d s^T (th = 2 pi kx / Nx), diagonalised on the host:
// Kx(kx) = Vx diag(lx) Vx^*, Ky(ky) = Vy diag(ly) Vy^*.  z~ = Ahat^+ r~ is then: a real DFT
// along x of the n^2 node fields and Vx^* per (cy, kx, a); a DFT along y, Vy^* per (ky, kx, j),
// division by ly_i + lx_j (the constant mode, the one pair whose sum is exactly 0, dropped),
// Vy and the inverse DFT along y; Vx and the inverse real DFT along x.  Three grid-wide phases
// over the spectrum S[kx][cy][a][j] (kx <= Nx/2).
enum : int { kPrecondJacobi = 0, kPrecondTwoLevel = 1, kPrecondSpectral = 2 };

template <typename T>
struct PrecondArgs {
  int kind;             // kPrecondTwoLevel or kPrecondSpectral
  const T* Bt;          // N^2 x N^2, row-major
  const Cplx<T>* twx;   // exp(-2 pi i m / Nx), m < Nx
  const Cplx<T>* twy;   // exp(-2 pi i m / Ny), m < Ny
  const T* ax;          // coarse eigenvalues: lambda(kx, ky) = ax[kx] + ay[ky]
  const T* ay;
  int log2x, log2y;     // log2 of Nx, Ny when powers of two, else -1 (direct DFT)
  T* z;                 // cell-block part of z~ (two-level) or all of z~ (spectral), one per dof
  T* rc;                // restricted residual (one per cell)
  T* uc;                // coarse correction (one per cell)
  Cplx<T>* C;           // coarse spectrum (Ny x (Nx/2 + 1))
  const Cplx<T>* Vx;    // spectral: Vx[kx][b][j], kx <= Nx/2 (column j = eigenvector j)
  const T* lx;          // lx[kx][j]
  const Cplx<T>* Vy;    // Vy[ky][a][i], ky < Ny
  const T* ly;          // ly[ky][i]
  Cplx<T>* S;           // spectrum, (Nx/2 + 1) x Ny x N x N
};

// Shared memory and synchronisation of one persistent solve.
template <typename T>
struct SolveCtx {
  T *sU, *tXR, *tXL, *tYR, *tYL;  // tile staging
  Cplx<T>* line0;                 // DFT line buffers (alias the tile staging)
  Cplx<T>* line1;
  const T* Bs;                    // Bt staged in shared memory (null without preconditioner)
  T* red;
  T* bcast;
  int* s_flag;
  SyncState* sync;
  T* part;                        // 6 * vsize: two alternating halves of up to 3 sums
  int phase;
  unsigned int tbase;             // first ticket of the next dynamically scheduled phase
  int vrank, vsize;               // this block's rank and the block count of the (virtual) grid
  int cluster;                    // the whole grid is one thread-block cluster
  // float32 solves: if kdf is set (an OpsK<df, N> in shared memory), the operator Ahat is
  // applied in double-float arithmetic on the float32 vectors, staged in the 8-byte tile
  // buffers wU, wXR, wXL, wYR, wYL (the float64 context's staging region)
  const void* kdf;
  df *wU, *wXR, *wXL, *wYR, *wYL;
};

// The barrier between the phases of a solve: the hardware cluster barrier when the solve's
// blocks form one cluster (small grids), else the capped grid barrier.
template <typename T>
__device__ __forceinline__ bool solve_barrier(SolveCtx<T>& X) {
  if (X.cluster) {
    cluster_barrier();
    return true;
  }
  return grid_barrier(X.sync, X.s_flag, X.vsize);
}

// Dynamic distribution of a phase's work units over the blocks of a solve: each block takes
// the next unit from the ticket counter of the solve's SyncState until the units run out.
// Every block draws exactly one ticket past the last unit, so a phase consumes units + vsize
// tickets and every block knows where the next phase's tickets start (X.tbase, read from
// the counter by every block at the start of the solve, before its first barrier).  Units
// write disjoint outputs, so the results do not depend on which block takes which unit.
template <typename T>
__device__ __forceinline__ int next_unit(SolveCtx<T>& X, int units) {
  int* s = reinterpret_cast<int*>(X.red);
  __syncthreads();  // every thread has read the previous unit number
  if (threadIdx.x == 0) s[0] = int(atomicAdd(&X.sync->ticket, 1u) - X.tbase);
  __syncthreads();
  return s[0];
}

template <typename T>
__device__ __forceinline__ void end_units(SolveCtx<T>& X, int units) {
  X.tbase += unsigned(units) + unsigned(X.vsize);
}

template <typename T>
__device__ __forceinline__ unsigned int read_ticket(const SyncState* s) {
  return *reinterpret_cast<const volatile unsigned int*>(&s->ticket);
}

// Block partials of one or two sums -> grid barrier -> the sums in every block (fixed order).
template <typename T>
__device__ __forceinline__ bool reduce_all(SolveCtx<T>& X, T v0, T& out0) {
  T* ph = X.part + (X.phase & 1) * 3 * X.vsize;
  ++X.phase;
  v0 = block_sum(v0, X.red);
  if (threadIdx.x == 0) __stcg(ph + X.vrank, v0);
  if (!solve_barrier(X)) return false;
  out0 = sum_partials_block(ph, X.vsize, 1, X.red, X.bcast);
  return true;
}

template <typename T>
__device__ __forceinline__ bool reduce_all2(SolveCtx<T>& X, T v0, T v1, T& out0, T& out1) {
  T* ph = X.part + (X.phase & 1) * 3 * X.vsize;
  ++X.phase;
  v0 = block_sum(v0, X.red);
  if (threadIdx.x == 0) __stcg(ph + 2 * X.vrank, v0);
  v1 = block_sum(v1, X.red);
  if (threadIdx.x == 0) __stcg(ph + 2 * X.vrank + 1, v1);
  if (!solve_barrier(X)) return false;
  out0 = sum_partials_block(ph, X.vsize, 2, X.red, X.bcast);
  out1 = sum_partials_block(ph + 1, X.vsize, 2, X.red, X.bcast);
  return true;
}

template <typename T>
__device__ __forceinline__ bool reduce_all3(SolveCtx<T>& X, T v0, T v1, T v2, T& out0, T& out1, T& out2) {
  T* ph = X.part + (X.phase & 1) * 3 * X.vsize;
  ++X.phase;
  v0 = block_sum(v0, X.red);
  if (threadIdx.x == 0) __stcg(ph + 3 * X.vrank, v0);
  v1 = block_sum(v1, X.red);
  if (threadIdx.x == 0) __stcg(ph + 3 * X.vrank + 1, v1);
  v2 = block_sum(v2, X.red);
  if (threadIdx.x == 0) __stcg(ph + 3 * X.vrank + 2, v2);
  if (!solve_barrier(X)) return false;
  out0 = sum_partials_block(ph, X.vsize, 3, X.red, X.bcast);
  out1 = sum_partials_block(ph + 1, X.vsize, 3, X.red, X.bcast);
  out2 = sum_partials_block(ph + 2, X.vsize, 3, X.red, X.bcast);
  return true;
}

// One CG tile pass: stage u = load(...) (plus-shaped halo), apply Ahat, hand (g, k, u, q)
// to out(...).
template <typename T, int N, class Tab, class LoadF, class OutF>
__device__ __forceinline__ void cg_tile_apply(const Tab& C, const Geom& G, int tile, SolveCtx<T>& X, LoadF&& load,
                                              OutF&& out) {
  constexpr int NN = N * N;
  const TileBox B = make_box(G, tile);
  stage_box<T, N>(G, B, X.sU, false, load);
  __syncthreads();
  line_traces<T, N>(B, X.sU, X.sU, C.kx, C.ky, X.tXR, X.tXL, X.tYR, X.tYL, false);
  __syncthreads();
  if (G.bc) {
    dirichlet_first_traces<T, N>(B, X.sU, X.sU, C.kx, C.ky, X.tXL, X.tYL);
    __syncthreads();
  }
  const int nin = B.TYe * B.TXe * NN;
  if constexpr (sizeof(T) == 4 && kThreads % NN == 0) {
    // float32: every node a thread visits is node k = threadIdx.x mod n^2 of its cell, so the
    // operator rows of that node are held in registers across the thread's cells (same
    // arithmetic and order as op_x_at / op_y_at)
    const int k = threadIdx.x % NN, a = k / N, b = k % N;
    T mx[N], my[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
      mx[j] = C.kx.M[b][j];
      my[j] = C.ky.M[a][j];
    }
    const T xa = C.kx.a[b], xd = C.kx.d[b], ya = C.ky.a[a], yd = C.ky.d[a];
    for (int i = threadIdx.x; i < nin; i += kThreads) {
      const int c = i / NN;
      const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
      const int lc = (ry + 1) * B.BW + rx + 1;
      const T* ux = X.sU + lc * (NN + 1) + a * N;
      const T* uy = X.sU + lc * (NN + 1) + b;
      T qx = xa * X.tXR[(lc + 1) * N + a];
      qx = fma(xd, X.tXL[(lc - 1) * N + a], qx);
      T qy = ya * X.tYR[(lc + B.BW) * N + b];
      qy = fma(yd, X.tYL[(lc - B.BW) * N + b], qy);
      if (G.bc && ((B.tx0 == 0 && rx == 0) || (B.ty0 == 0 && ry == 0))) {  // a Dirichlet boundary cell
        const bool fx = B.tx0 + rx == 0, fy = B.ty0 + ry == 0;
        const T* Mx = fx ? C.kx.Mf[b] : C.kx.M[b];
        const T* My = fy ? C.ky.Mf[a] : C.ky.M[a];
        qx = (fx ? C.kx.af[b] : xa) * X.tXR[(lc + 1) * N + a];
        qx = fma(xd, X.tXL[(lc - 1) * N + a], qx);
        qy = (fy ? C.ky.af[a] : ya) * X.tYR[(lc + B.BW) * N + b];
        qy = fma(yd, X.tYL[(lc - B.BW) * N + b], qy);
#pragma unroll
        for (int j = 0; j < N; ++j) qx = fma(Mx[j], ux[j], qx);
#pragma unroll
        for (int j = 0; j < N; ++j) qy = fma(My[j], uy[j * N], qy);
      } else {
#pragma unroll
        for (int j = 0; j < N; ++j) qx = fma(mx[j], ux[j], qx);
#pragma unroll
        for (int j = 0; j < N; ++j) qy = fma(my[j], uy[j * N], qy);
      }
      const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
      out(g, k, X.sU[lc * (NN + 1) + k], qx + qy);
    }
  } else {
    if (!G.bc) {
      for (int i = threadIdx.x; i < nin; i += blockDim.x) {
        const int c = i / NN, k = i - (i / NN) * NN;
        const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
        const int lc = (ry + 1) * B.BW + rx + 1;
        const int a = k / N, b = k - (k / N) * N;
        const T q = op_x_at<T, N>(X.sU, X.tXR, X.tXL, C.kx, lc, a, b) +
                    op_y_at<T, N>(X.sU, X.tYR, X.tYL, C.ky, lc, B.BW, a, b);
        const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
        out(g, k, X.sU[lc * (NN + 1) + k], q);
      }
    } else {  // Dirichlet: the first cell of a line takes its own blocks (Op1D::Mf, af)
      for (int i = threadIdx.x; i < nin; i += blockDim.x) {
        const int c = i / NN, k = i - (i / NN) * NN;
        const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
        const int lc = (ry + 1) * B.BW + rx + 1;
        const int a = k / N, b = k - (k / N) * N;
        const bool fx = B.tx0 + rx == 0, fy = B.ty0 + ry == 0;
        const T q = op_x_at<T, N>(X.sU, X.tXR, X.tXL, C.kx, lc, a, b, fx) +
                    op_y_at<T, N>(X.sU, X.tYR, X.tYL, C.ky, lc, B.BW, a, b, fy);
        const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
        out(g, k, X.sU[lc * (NN + 1) + k], q);
      }
    }
  }
  __syncthreads();
}

// One tile pass of the solve's operator: cg_tile_apply in T, or -- for a float32 solve with
// the compensated apply enabled -- in double-float arithmetic on the same float32 values, the
// result rounded to float32.  A float32 evaluation of Ahat u has an absolute error of about
// eps32 |Ahat| |u|, which on the smoothest modes of a fine grid (eigenvalue ~1 against
// |Ahat| ~ 1e7 at 1024^2 cells, n = 5) is as large as Ahat u itself; the double-float apply
// brings it down to ~eps32^2 |Ahat| |u|.
template <typename T, int N, class LoadF, class OutF>
__device__ __forceinline__ void solve_apply(const Ops2D<T, N>& C, const Geom& G, int tile, SolveCtx<T>& X,
                                            LoadF&& load, OutF&& out) {
  if constexpr (std::is_same<T, float>::value) {
    if (X.kdf) {
      SolveCtx<df> W;
      W.sU = X.wU;
      W.tXR = X.wXR;
      W.tXL = X.wXL;
      W.tYR = X.wYR;
      W.tYL = X.wYL;
      cg_tile_apply<df, N>(
          *static_cast<const OpsK<df, N>*>(X.kdf), G, tile, W,
          [&](size_t g, int k, bool interior) { return df(load(g, k, interior)); },
          [&](size_t g, int k, df u, df q) { out(g, k, u.hi, to_float(q)); });
      return;
    }
  }
  cg_tile_apply<T, N>(C, G, tile, X, load, out);
}

// Where the tile's residual is staged for the preconditioner's cell part: X.sU itself, or,
// with a float32 preconditioner in a float64 solve, a float32 copy in the (then unused) trace
// arrays.
template <typename T, typename TP>
__device__ __forceinline__ TP* pc_stage(SolveCtx<T>& X) {
  if constexpr (std::is_same<T, TP>::value)
    return X.sU;
  else
    return reinterpret_cast<TP*>(X.tXR);
}

// Cell part of the preconditioner on one tile whose interior residual is staged (X.sU, and its
// copy in the preconditioner's precision TP): z~ = Bt r~ on every cell, rc = sum sqrt(W) r~ per
// cell (to P.rc); returns the tile's r~ . z~_block (in T).
template <typename T, int N, typename TP = T>
__device__ __forceinline__ T pc_cells(const Ops2D<T, N>& C, const Geom& G, const TileBox& B,
                                      const PrecondArgs<TP>& P, SolveCtx<T>& X) {
  constexpr int NN = N * N;
  const TP* Bs = reinterpret_cast<const TP*>(X.Bs);
  const TP* su = pc_stage<T, TP>(X);
  T rz = T(0);
  const int nin = B.TYe * B.TXe * NN;
  if constexpr (sizeof(TP) == 4 && kThreads % NN == 0) {
    // float32: a thread's nodes all have k = threadIdx.x mod n^2, so its column of Bt stays in
    // registers (same arithmetic and order as below)
    const int k = threadIdx.x % NN;
    TP bk[NN];
#pragma unroll
    for (int j = 0; j < NN; ++j) bk[j] = Bs[j * NN + k];
    for (int i = threadIdx.x; i < nin; i += kThreads) {
      const int c = i / NN;
      const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
      const int cell = ((ry + 1) * B.BW + rx + 1) * (NN + 1);
      const TP* u = su + cell;
      TP zj = TP(0);
#pragma unroll
      for (int j = 0; j < NN; ++j) zj = fma(bk[j], u[j], zj);
      const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
      __stcg(P.z + g, zj);
      rz = fma(X.sU[cell + k], T(zj), rz);
    }
  } else {
    for (int i = threadIdx.x; i < nin; i += blockDim.x) {
      const int c = i / NN, k = i - (i / NN) * NN;
      const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
      const int cell = ((ry + 1) * B.BW + rx + 1) * (NN + 1);
      const TP* u = su + cell;
      TP zj = TP(0);
#pragma unroll
      for (int j = 0; j < NN; ++j) zj = fma(Bs[j * NN + k], u[j], zj);  // Bt is symmetric
      const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
      __stcg(P.z + g, zj);
      rz = fma(X.sU[cell + k], T(zj), rz);
    }
  }
  const int ncell = B.TYe * B.TXe;
  for (int c = threadIdx.x; c < ncell; c += blockDim.x) {
    const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
    const TP* u = su + ((ry + 1) * B.BW + rx + 1) * (NN + 1);
    TP v = TP(0);
#pragma unroll
    for (int k = 0; k < NN; ++k) v = fma(TP(C.sw[k]), u[k], v);
    __stcg(P.rc + (size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx), v);
  }
  return rz;
}

template <typename T>
__device__ __forceinline__ Cplx<T> ld_cplx(const Cplx<T>* p) {
  return Cplx<T>{__ldcg(&p->re), __ldcg(&p->im)};
}

// An entry of the spectral preconditioner's n x n transforms.  In float64 through the
// read-only path (the compiler then keeps them out of registers: holding a whole float64
// transform per direction would spill); in float32 a plain load (measured faster).
template <typename T>
__device__ __forceinline__ Cplx<T> ld_table(const Cplx<T>* p) {
  if constexpr (sizeof(T) == 8)
    return Cplx<T>{__ldg(&p->re), __ldg(&p->im)};
  else
    return *p;
}

template <typename T>
__device__ __forceinline__ void st_cplx(Cplx<T>* p, Cplx<T> v) {
  __stcg(&p->re, v.re);
  __stcg(&p->im, v.im);
}

// Coarse solve uc = A_c^+ rc (rc real, one value per cell).  Two real rows a, b travel as
// one complex row a + i b: its DFT Z gives both spectra, A_k = (Z_k + conj Z_-k) / 2 and
// B_k = (Z_k - conj Z_-k) / 2i, of which the columns kx = 0 .. Nx/2 are kept (the others are
// their conjugates).  Then per kept column: DFT over y, division by the eigenvalues (the
// constant mode dropped), inverse DFT; finally per row pair the inverse DFT of
// A + i B (extended by conjugate symmetry) returns row a in the real and row b in the
// imaginary part.  Three grid-wide phases; the spectrum array holds Ny x (Nx/2 + 1) values.
// Returns sum uc . rc (in every block).
template <typename T, typename TR = T>
__device__ __forceinline__ bool pc_coarse(const Geom& G, const PrecondArgs<T>& P, SolveCtx<TR>& X, TR& ucrc) {
  const int Nx = G.Nx, Ny = G.Ny;
  Cplx<T>* L0 = reinterpret_cast<Cplx<T>*>(X.line0);  // the solve's DFT line buffers, in T
  Cplx<T>* L1 = reinterpret_cast<Cplx<T>*>(X.line1);
  const int Nh = Nx / 2, W = Nh + 1;  // kept columns
  const int npairs = (Ny + 1) / 2;
  for (int pr = X.vrank; pr < npairs; pr += X.vsize) {
    const int ra = 2 * pr, rb = 2 * pr + 1;
    const bool hasb = rb < Ny;
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) {
      const T va = __ldcg(P.rc + (size_t)ra * Nx + j);
      const T vb = hasb ? __ldcg(P.rc + (size_t)rb * Nx + j) : T(0);
      L0[dft_slot(j, P.log2x)] = Cplx<T>{va, vb};
    }
    __syncthreads();
    dft_line(L0, L1, Nx, P.log2x, P.twx, false);
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
      const Cplx<T> zk = L0[k], zm = L0[k == 0 ? 0 : Nx - k];
      st_cplx(&P.C[(size_t)ra * W + k], Cplx<T>{T(0.5) * (zk.re + zm.re), T(0.5) * (zk.im - zm.im)});
      if (hasb) st_cplx(&P.C[(size_t)rb * W + k], Cplx<T>{T(0.5) * (zk.im + zm.im), T(0.5) * (zm.re - zk.re)});
    }
    __syncthreads();
  }
  if (!solve_barrier(X)) return false;
  const T scale = T(1) / (T(Nx) * T(Ny));
  for (int col = X.vrank; col < W; col += X.vsize) {
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) L0[dft_slot(j, P.log2y)] = ld_cplx(&P.C[(size_t)j * W + col]);
    __syncthreads();
    dft_line(L0, L1, Ny, P.log2y, P.twy, false);
    for (int ky = threadIdx.x; ky < Ny; ky += blockDim.x) {
      const T f = (col == 0 && ky == 0) ? T(0) : scale / (P.ax[col] + P.ay[ky]);
      const Cplx<T> v = L0[ky];
      L1[dft_slot(ky, P.log2y)] = Cplx<T>{v.re * f, v.im * f};
    }
    __syncthreads();
    dft_line(L1, L0, Ny, P.log2y, P.twy, true);
    for (int j = threadIdx.x; j < Ny; j += blockDim.x) st_cplx(&P.C[(size_t)j * W + col], L1[j]);
    __syncthreads();
  }
  if (!solve_barrier(X)) return false;
  TR acc = TR(0);
  for (int pr = X.vrank; pr < npairs; pr += X.vsize) {
    const int ra = 2 * pr, rb = 2 * pr + 1;
    const bool hasb = rb < Ny;
    for (int k = threadIdx.x; k < Nx; k += blockDim.x) {
      // A_k, B_k for k > Nx/2 are the conjugates of the kept columns Nx - k
      const bool kept = k < W;
      const int kk = kept ? k : Nx - k;
      Cplx<T> A = ld_cplx(&P.C[(size_t)ra * W + kk]);
      Cplx<T> B = hasb ? ld_cplx(&P.C[(size_t)rb * W + kk]) : Cplx<T>{T(0), T(0)};
      if (!kept) {
        A.im = -A.im;
        B.im = -B.im;
      }
      L0[dft_slot(k, P.log2x)] = Cplx<T>{A.re - B.im, A.im + B.re};
    }
    __syncthreads();
    dft_line(L0, L1, Nx, P.log2x, P.twx, true);
    for (int j = threadIdx.x; j < Nx; j += blockDim.x) {
      const size_t ca = (size_t)ra * Nx + j;
      const T ua = L0[j].re;
      __stcg(P.uc + ca, ua);
      acc = fma(TR(ua), TR(__ldcg(P.rc + ca)), acc);
      if (hasb) {
        const size_t cb = (size_t)rb * Nx + j;
        const T ub = L0[j].im;
        __stcg(P.uc + cb, ub);
        acc = fma(TR(ub), TR(__ldcg(P.rc + cb)), acc);
      }
    }
    __syncthreads();
  }
  return reduce_all(X, acc, ucrc);
}

// ---- the spectral preconditioner's three phases (see PrecondArgs) -------------------------
// Units of the row phases: (row pair pr, node row a): rows cy0 = 2 pr, cy1 = 2 pr + 1 travel as
// one complex line per node column b (real part row cy0, imaginary part row cy1), as in
// pc_coarse.  Shared memory: N lines of max(Nx, Ny) complex values (twice that for the direct
// DFT of a length that is not a power of two).

// Phase 1: S[kx][cy][a][j] = sum_b conj(Vx[kx][b][j]) DFT_x(r~[cy, ., a, b])[kx].
template <typename TP, int N, typename TR>
__device__ __forceinline__ void spectral_rows_fwd(const Geom& G, const PrecondArgs<TP>& P, const TR* r,
                                                  SolveCtx<TR>& X) {
  const int Nx = G.Nx, Ny = G.Ny, W = Nx / 2 + 1;
  Cplx<TP>* L0 = reinterpret_cast<Cplx<TP>*>(X.line0);
  Cplx<TP>* Lt = L0 + N * Nx;
  const int units = (Ny + 1) / 2 * N;
  for (int u = next_unit(X, units); u < units; u = next_unit(X, units)) {
    const int pr = u / N, a = u - pr * N;
    const int cy0 = 2 * pr, cy1 = cy0 + 1;
    const bool hasb = cy1 < Ny;
    for (int i = threadIdx.x; i < Nx * N; i += blockDim.x) {
      const int cx = i / N, b = i - cx * N;
      const TP va = TP(__ldcg(r + (((size_t)cy0 * Nx + cx) * N + a) * N + b));
      const TP vb = hasb ? TP(__ldcg(r + (((size_t)cy1 * Nx + cx) * N + a) * N + b)) : TP(0);
      L0[b * Nx + dft_slot(cx, P.log2x)] = Cplx<TP>{va, vb};
    }
    __syncthreads();
    fft_lines(L0, Lt, N, Nx, P.log2x, P.twx, false, false);
#pragma unroll 1
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
      const int km = k == 0 ? 0 : Nx - k;
      Cplx<TP> A[N], B[N];
#pragma unroll
      for (int b = 0; b < N; ++b) {
        const Cplx<TP> zk = L0[b * Nx + k], zm = L0[b * Nx + km];
        A[b] = Cplx<TP>{TP(0.5) * (zk.re + zm.re), TP(0.5) * (zk.im - zm.im)};
        B[b] = Cplx<TP>{TP(0.5) * (zk.im + zm.im), TP(0.5) * (zm.re - zk.re)};
      }
      const Cplx<TP>* V = P.Vx + (size_t)k * N * N;
      Cplx<TP>* Sa = P.S + (((size_t)k * Ny + cy0) * N + a) * N;
      Cplx<TP>* Sb = P.S + (((size_t)k * Ny + cy1) * N + a) * N;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        Cplx<TP> ta{TP(0), TP(0)}, tb{TP(0), TP(0)};
#pragma unroll
        for (int b = 0; b < N; ++b) {
          const Cplx<TP> v = ld_table(V + b * N + j);  // conj(v) * x
          ta.re = fma(v.re, A[b].re, fma(v.im, A[b].im, ta.re));
          ta.im = fma(v.re, A[b].im, fma(-v.im, A[b].re, ta.im));
          tb.re = fma(v.re, B[b].re, fma(v.im, B[b].im, tb.re));
          tb.im = fma(v.re, B[b].im, fma(-v.im, B[b].re, tb.im));
        }
        st_cplx(Sa + j, ta);
        if (hasb) st_cplx(Sb + j, tb);
      }
    }
    __syncthreads();
  }
  end_units(X, units);
}

// Phase 2, per unit (kx, j): DFT along y of S[kx][.][a][j] for every a, then per ky
// t = Vy^* x, t_i *= scale / (ly_i + lx_j) (0 for the constant mode), x = Vy t, inverse DFT.
template <typename TP, int N, typename TR>
__device__ __forceinline__ void spectral_cols(const Geom& G, const PrecondArgs<TP>& P, SolveCtx<TR>& X) {
  const int Nx = G.Nx, Ny = G.Ny, W = Nx / 2 + 1;
  Cplx<TP>* L0 = reinterpret_cast<Cplx<TP>*>(X.line0);
  Cplx<TP>* Lt = L0 + N * Ny;
  const TP scale = TP(1) / (TP(Nx) * TP(Ny));
  for (int u = next_unit(X, W * N); u < W * N; u = next_unit(X, W * N)) {
    const int kx = u / N, j = u - kx * N;
    const Cplx<TP>* Sk = P.S + (size_t)kx * Ny * N * N;
    for (int i = threadIdx.x; i < Ny * N; i += blockDim.x) {
      const int cy = i / N, a = i - cy * N;
      L0[a * Ny + dft_slot(cy, P.log2y)] = ld_cplx(Sk + ((size_t)cy * N + a) * N + j);
    }
    __syncthreads();
    fft_lines(L0, Lt, N, Ny, P.log2y, P.twy, false, false);
    const TP lxj = P.lx[kx * N + j];
#pragma unroll 1
    for (int ky = threadIdx.x; ky < Ny; ky += blockDim.x) {
      const Cplx<TP>* V = P.Vy + (size_t)ky * N * N;
      Cplx<TP> t[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        Cplx<TP> acc{TP(0), TP(0)};
#pragma unroll
        for (int a = 0; a < N; ++a) {
          const Cplx<TP> v = ld_table(V + a * N + i), x = L0[a * Ny + ky];
          acc.re = fma(v.re, x.re, fma(v.im, x.im, acc.re));
          acc.im = fma(v.re, x.im, fma(-v.im, x.re, acc.im));
        }
        const TP den = P.ly[ky * N + i] + lxj;
        const TP f = den == TP(0) ? TP(0) : scale / den;
        t[i] = Cplx<TP>{acc.re * f, acc.im * f};
      }
#pragma unroll
      for (int a = 0; a < N; ++a) {
        Cplx<TP> acc{TP(0), TP(0)};
#pragma unroll
        for (int i = 0; i < N; ++i) acc = cadd(acc, cmul(ld_table(V + a * N + i), t[i]));
        L0[a * Ny + ky] = acc;
      }
    }
    __syncthreads();
    fft_lines(L0, Lt, N, Ny, P.log2y, P.twy, true, true);
    Cplx<TP>* Sw = P.S + (size_t)kx * Ny * N * N;
    for (int i = threadIdx.x; i < Ny * N; i += blockDim.x) {
      const int cy = i / N, a = i - cy * N;
      st_cplx(Sw + ((size_t)cy * N + a) * N + j, L0[a * Ny + dft_slot(cy, P.log2y)]);
    }
    __syncthreads();
  }
  end_units(X, W * N);
}

// Phase 3: z~[cy, ., a, b] = inverse real DFT_x of sum_j Vx[kx][b][j] S[kx][cy][a][j].
template <typename TP, int N, typename TR>
__device__ __forceinline__ void spectral_rows_inv(const Geom& G, const PrecondArgs<TP>& P, SolveCtx<TR>& X) {
  const int Nx = G.Nx, Ny = G.Ny, W = Nx / 2 + 1;
  Cplx<TP>* L0 = reinterpret_cast<Cplx<TP>*>(X.line0);
  Cplx<TP>* Lt = L0 + N * Nx;
  const int units = (Ny + 1) / 2 * N;
  for (int u = next_unit(X, units); u < units; u = next_unit(X, units)) {
    const int pr = u / N, a = u - pr * N;
    const int cy0 = 2 * pr, cy1 = cy0 + 1;
    const bool hasb = cy1 < Ny;
#pragma unroll 1
    for (int k = threadIdx.x; k < W; k += blockDim.x) {
      const Cplx<TP>* V = P.Vx + (size_t)k * N * N;
      const Cplx<TP>* Sa = P.S + (((size_t)k * Ny + cy0) * N + a) * N;
      const Cplx<TP>* Sb = P.S + (((size_t)k * Ny + cy1) * N + a) * N;
      Cplx<TP> ta[N], tb[N];
#pragma unroll
      for (int j = 0; j < N; ++j) {
        ta[j] = ld_cplx(Sa + j);
        tb[j] = hasb ? ld_cplx(Sb + j) : Cplx<TP>{TP(0), TP(0)};
      }
      const bool mirror = k > 0 && 2 * k != Nx;  // Nx - k is a distinct bin
#pragma unroll
      for (int b = 0; b < N; ++b) {
        Cplx<TP> A{TP(0), TP(0)}, B{TP(0), TP(0)};
#pragma unroll
        for (int j = 0; j < N; ++j) {
          const Cplx<TP> v = ld_table(V + b * N + j);
          A = cadd(A, cmul(v, ta[j]));
          B = cadd(B, cmul(v, tb[j]));
        }
        // Z = A + i B at k; at Nx - k the spectra of the real rows are conj(A), conj(B)
        L0[b * Nx + k] = Cplx<TP>{A.re - B.im, A.im + B.re};
        if (mirror) L0[b * Nx + Nx - k] = Cplx<TP>{A.re + B.im, B.re - A.im};
      }
    }
    __syncthreads();
    fft_lines(L0, Lt, N, Nx, P.log2x, P.twx, true, true);
    for (int i = threadIdx.x; i < Nx * N; i += blockDim.x) {
      const int cx = i / N, b = i - cx * N;
      const Cplx<TP> zv = L0[b * Nx + dft_slot(cx, P.log2x)];
      __stcg(P.z + (((size_t)cy0 * Nx + cx) * N + a) * N + b, zv.re);
      if (hasb) __stcg(P.z + (((size_t)cy1 * Nx + cx) * N + a) * N + b, zv.im);
    }
    __syncthreads();
  }
  end_units(X, units);
}

// z~ = Ahat^+ r~ (spectral preconditioner): the three phases and the sum r~ . z~ (in every block).
template <typename TP, int N, typename TR>
__device__ __forceinline__ bool pc_spectral(const Geom& G, const PrecondArgs<TP>& P, const TR* r, SolveCtx<TR>& X,
                                            TR& rz) {
  spectral_rows_fwd<TP, N, TR>(G, P, r, X);
  if (!solve_barrier(X)) return false;
  spectral_cols<TP, N, TR>(G, P, X);
  if (!solve_barrier(X)) return false;
  spectral_rows_inv<TP, N, TR>(G, P, X);
  if (!solve_barrier(X)) return false;
  // r~ . z~ in a fixed order over the dofs (the units above were scheduled dynamically)
  const size_t ndof = (size_t)G.Nx * G.Ny * N * N;
  TR acc = TR(0);
  for (size_t i = (size_t)X.vrank * blockDim.x + threadIdx.x; i < ndof; i += (size_t)X.vsize * blockDim.x)
    acc = fma(TR(__ldcg(P.z + i)), __ldcg(r + i), acc);
  return reduce_all(X, acc, rz);
}

// z~ = M^-1 r~ for the residual currently in r; returns r~ . z~ in rz.
template <typename T, int N, typename TP = T>
__device__ __forceinline__ bool pc_apply(const Ops2D<T, N>& C, const Geom& G, const PrecondArgs<TP>& P, const T* r,
                                         SolveCtx<T>& X, T& rz) {
  constexpr int NN = N * N;
  if (P.kind == kPrecondSpectral) return pc_spectral<TP, N, T>(G, P, r, X, rz);
  const int ntiles = G.tilesX * G.tilesY;
  TP* su = pc_stage<T, TP>(X);
  T rzb = T(0);
  for (int t = X.vrank; t < ntiles; t += X.vsize) {
    const TileBox B = make_box(G, t);
    const int nin = B.TYe * B.TXe * NN;
    for (int i = threadIdx.x; i < nin; i += blockDim.x) {
      const int c = i / NN, k = i - (i / NN) * NN;
      const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
      const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
      const int o = ((ry + 1) * B.BW + rx + 1) * (NN + 1) + k;
      const T v = __ldcg(r + g);
      X.sU[o] = v;
      if constexpr (!std::is_same<T, TP>::value) su[o] = TP(v);
    }
    __syncthreads();
    rzb += pc_cells<T, N, TP>(C, G, B, P, X);
    __syncthreads();
  }
  T rzsum = T(0);
  if (!reduce_all(X, rzb, rzsum)) return false;
  T ucrc = T(0);
  if (!pc_coarse<TP, T>(G, P, X, ucrc)) return false;
  rz = rzsum + ucrc;
  return true;
}

// The CG iterations proper (PCG when P is non-null), from r (residual of the current y) with
// rr = r.r, rhob = b.b (the stopping rule is on r.r) and, with a preconditioner, z = M^-1 r
// already applied and rz = r.z.  The stopping rule is on the true residual: when the
// recursive residual meets the tolerance, one more tile pass computes b - Ahat y; if that
// misses the tolerance, CG restarts from it.  Returns the iteration count; raises flags.
template <typename T, int N, typename TP = T>
__device__ __forceinline__ int cg_iterate(const Ops2D<T, N>& C, const Geom& G, const CgVectors<T>& V,
                                          const PrecondArgs<TP>* P, const RhsSource<T>& Bsrc, SolveCtx<T>& X,
                                          T& rr, T rz, T rhob, double tol2, int maxit, int fixed_iters, int& flags,
                                          int max_restarts = kMaxRestarts, double floor2 = 0.0, T* ay = nullptr) {
  constexpr int NN = N * N;
  const int ntiles = G.tilesX * G.tilesY;
  const size_t ndof = (size_t)G.Nx * G.Ny * NN;
  const size_t stride = (size_t)X.vsize * blockDim.x;
  int it = 0, restarts = 0;
  double rr_prev = -1.0;  // true residual at the previous verification
  T beta = T(0);
  int cur = 0;
  bool first = true;  // p = z (no previous direction)
  const bool spec = P && P->kind == kPrecondSpectral;
  if (!P) rz = rr;
  while (true) {
    if (fixed_iters > 0) {
      if (it >= fixed_iters) break;
    } else if (double(rr) <= tol2 * double(rhob)) {
      if (max_restarts == 0) break;  // loose inner solves: the recursive residual suffices
      // Verify on the true residual r = b - Ahat y: accept it below the tolerance, or once it
      // stagnates below the float64 rounding floor of the iterate y (floor2 * y.y, see
      // CgArgs::floor2), where no float64 iterate can do better.
      T rt = T(0), yt = T(0);
      for (int t = X.vrank; t < ntiles; t += X.vsize) {
        solve_apply<T, N>(
            C, G, t, X, [&](size_t g, int, bool) { return __ldcg(V.y + g); },
            [&](size_t g, int k, T yv, T qv) {
              const T r = rhs_at<T, N>(C, Bsrc, g, k) - qv;
              __stcg(V.r + g, r);
              if (ay) __stcg(ay + g, qv);
              rt = fma(r, r, rt);
              yt = fma(yv, yv, yt);
            });
      }
      T rr_true = T(0), yy = T(0);
      if (!reduce_all2(X, rt, yt, rr_true, yy)) {
        flags |= kFlagTimeout;
        return it;
      }
      rr = rr_true;
      if (double(rr_true) <= tol2 * double(rhob)) break;
      // stagnation at the rounding floor: below it, and less than a factor 4 below the previous
      // check's true residual
      if (double(rr_true) <= floor2 * double(yy) && rr_prev >= 0.0 && double(rr_true) > 0.25 * rr_prev) break;
      rr_prev = double(rr_true);
      if (restarts >= max_restarts) {
        flags |= kFlagNoconv;
        break;
      }
      ++restarts;
      if (P) {
        if (!pc_apply<T, N, TP>(C, G, *P, V.r, X, rz)) {
          flags |= kFlagTimeout;
          return it;
        }
      } else {
        rz = rr;
      }
      first = true;
      continue;
    }
    if (rr == T(0)) break;
    if (it >= maxit) {
      flags |= kFlagNoconv;
      break;
    }
    T* pin = cur ? V.p1 : V.p0;
    T* pout = cur ? V.p0 : V.p1;
    // Phase A: p = z + beta p_old (halo recomputed locally), q = Ahat p, p.q.
    T pq = T(0);
    for (int t = X.vrank; t < ntiles; t += X.vsize) {
      solve_apply<T, N>(
          C, G, t, X,
          [&](size_t g, int k, bool interior) {
            const T zv = spec ? T(__ldcg(P->z + g))
                         : P  ? fma(C.sw[k], T(__ldcg(P->uc + g / NN)), T(__ldcg(P->z + g)))
                              : __ldcg(V.r + g);
            const T pv = first ? zv : fma(beta, __ldcg(pin + g), zv);
            if (interior) __stcg(pout + g, pv);
            return pv;
          },
          [&](size_t g, int, T pv, T qv) {
            __stcg(V.q + g, qv);
            pq = fma(pv, qv, pq);
          });
    }
    T pqs = T(0);
    if (!reduce_all(X, pq, pqs)) {
      flags |= kFlagTimeout;
      return it;
    }
    if (!(pqs > T(0))) {
      // In parity mode (a fixed iteration count) CG may run past exact convergence on tiny
      // systems, where p.q is rounding noise (zero or negative): stop there.  Anything else
      // (a non-positive p.q in a tolerance-stopped solve, or NaN) is a breakdown.
      if (!(fixed_iters > 0 && pqs <= T(0))) flags |= kFlagBreakdown;
      break;
    }
    const T alpha = rz / pqs;
    // Phase B: y += alpha p, r -= alpha q, r.r (and the cell part of the preconditioner).
    T rrb = T(0), rzb = T(0);
    if (!P || spec) {
      struct Pqyr {
        T p, q, y, r;
      };
      strided_pass<2>(
          (size_t)X.vrank * blockDim.x + threadIdx.x, ndof, stride,
          [&](size_t i) { return Pqyr{__ldcg(pout + i), __ldcg(V.q + i), __ldcg(V.y + i), __ldcg(V.r + i)}; },
          [&](size_t i, const Pqyr& v) {
            const T yv = fma(alpha, v.p, v.y);
            const T rv = fma(-alpha, v.q, v.r);
            __stcg(V.y + i, yv);
            __stcg(V.r + i, rv);
            rrb = fma(rv, rv, rrb);
          });
    } else {
      for (int t = X.vrank; t < ntiles; t += X.vsize) {
        const TileBox B = make_box(G, t);
        const int nin = B.TYe * B.TXe * NN;
        for (int i = threadIdx.x; i < nin; i += blockDim.x) {
          const int c = i / NN, k = i - (i / NN) * NN;
          const int ry = quot(c, B.mTXe), rx = c - ry * B.TXe;
          const size_t g = ((size_t)(B.ty0 + ry) * G.Nx + (B.tx0 + rx)) * NN + k;
          const T pv = __ldcg(pout + g), qv = __ldcg(V.q + g);
          const T yv = fma(alpha, pv, __ldcg(V.y + g));
          const T rv = fma(-alpha, qv, __ldcg(V.r + g));
          __stcg(V.y + g, yv);
          __stcg(V.r + g, rv);
          rrb = fma(rv, rv, rrb);
          const int o = ((ry + 1) * B.BW + rx + 1) * (NN + 1) + k;
          X.sU[o] = rv;
          if constexpr (!std::is_same<T, TP>::value) pc_stage<T, TP>(X)[o] = TP(rv);
        }
        __syncthreads();
        rzb += pc_cells<T, N, TP>(C, G, B, *P, X);
        __syncthreads();
      }
    }
    T rnew = T(0), rzjs = T(0);
    if (!reduce_all2(X, rrb, rzb, rnew, rzjs)) {
      flags |= kFlagTimeout;
      return it;
    }
    T rznew = rnew;
    if (fixed_iters == 0 && double(rnew) <= tol2 * double(rhob)) {
      // converged by the recursive residual: the next pass verifies the true residual and, on
      // a restart, preconditions that one, so this residual needs no preconditioning
      rr = rnew;
      cur ^= 1;
      first = false;
      ++it;
      continue;
    }
    if (spec) {
      if (!pc_spectral<TP, N, T>(G, *P, V.r, X, rznew)) {
        flags |= kFlagTimeout;
        return it;
      }
    } else if (P) {
      T ucrc = T(0);
      if (!pc_coarse<TP, T>(G, *P, X, ucrc)) {
        flags |= kFlagTimeout;
        return it;
      }
      rznew = rzjs + ucrc;
    }
    beta = rznew / rz;
    rz = rznew;
    rr = rnew;
    cur ^= 1;
    first = false;
    ++it;
  }
  return it;
}

// Removes the W-mean of psi = y / sqrt(W) from y (y -= m sqrt(W)): a preconditioner other
// than W^-1 moves the iterates along the constants, the kernel of A.
template <typename T, int N>
__device__ __forceinline__ bool project_mean(const Ops2D<T, N>& C, const Geom& G, T* y, double sumW,
                                             SolveCtx<T>& X) {
  constexpr int NN = N * N;
  const size_t ndof = (size_t)G.Nx * G.Ny * NN;
  const size_t stride = (size_t)X.vsize * blockDim.x;
  const size_t first = (size_t)X.vrank * blockDim.x + threadIdx.x;
  T s = T(0);
  strided_pass<4>(first, ndof, stride, [&](size_t i) { return __ldcg(y + i); },
                  [&](size_t i, T v) { s = fma(C.sw[i % NN], v, s); });
  T m = T(0);
  if (!reduce_all(X, s, m)) return false;
  m = m / T(sumW);
  strided_pass<4>(first, ndof, stride, [&](size_t i) { return __ldcg(y + i); },
                  [&](size_t i, T v) { __stcg(y + i, fma(-m, C.sw[i % NN], v)); });
  return solve_barrier(X);
}

template <typename T, typename TP = T>
struct CgArgs {
  const double* omega;  // b = sqrt(W) (omega - mean_W omega) ...
  const T* rhs;         // ... or b = rhs (scaled space) when non-null
  const double* xa;     // initial guess y0 = ca xa + cb xb (null terms dropped), times
  const double* xb;     // sqrt(W) when x_unscaled
  double ca, cb;
  int x_unscaled;
  // Recycled operator products (the stepper's extrapolated guesses): with axa non-null, Ahat y0
  // = ca axa + cb axb (scaled space, x_unscaled == 0) replaces the setup's operator application,
  // and with ay non-null the solve stores Ahat y of its final iterate there (from the verifying
  // true-residual pass that ends every tolerance-stopped solve).
  const T* axa;
  const T* axb;
  T* ay;
  CgVectors<T> v;
  int precond;          // kPrecondJacobi (W^-1: plain CG on the scaled system), kPrecondTwoLevel or kPrecondSpectral
  PrecondArgs<TP> pc;   // (TP = float: the preconditioner applied in float32)
  double* psi_out;      // if non-null: psi = y / sqrt(W) at the end
  T* part;              // 6 * gridDim.x
  SyncState* sync;
  SolveStatus* status;
  double tol2;
  // The float64 rounding floor of the residual, per unit y.y: rounding y to float64 and
  // evaluating b - Ahat y in float64 leave a residual of up to about 2 u lambda_max |y|
  // (u = 2^-53, lambda_max bounded by the row sums of |Ahat|), so floor2 = (2^-52 lambda)^2;
  // a solve whose true residual stagnates below floor2 y.y stops there, even above tol2 b.b.
  double floor2;
  int maxit, fixed_iters;
  double sumW;
  int cluster;          // launched as one thread-block cluster (cluster barriers)
  int keep_mean;        // homogeneous Dirichlet: A is definite, b = sqrt(W) omega (no mean removed)
};

// Dynamic shared memory of the persistent solves: [Bt (with the preconditioner)] then one
// region used both for the tile staging and for two DFT lines.
__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T, int N>
__host__ __device__ constexpr size_t cg_tile_values(int TY, int TX) {
  return (size_t)(TY + 2) * (TX + 2) * (N * N + 1 + 4 * N);
}

// Bytes of the DFT line buffers of a preconditioner (kind: PrecondArgs): two lines for the
// two-level coarse solve, N lines (2N for a length that is not a power of two) for the spectral
// one; pow2: both cell counts are powers of two.
template <typename T, int N>
__host__ __device__ constexpr size_t pc_line_bytes(int kind, int Lmax, bool pow2) {
  return kind == kPrecondTwoLevel   ? 2 * (size_t)Lmax * sizeof(Cplx<T>)
         : kind == kPrecondSpectral ? (pow2 ? 1 : 2) * (size_t)N * Lmax * sizeof(Cplx<T>)
                                    : 0;
}

template <typename T, int N>
__host__ __device__ constexpr size_t cg_smem_bytes(int TY, int TX, int Lmax, int kind, bool pow2) {
  return (kind == kPrecondTwoLevel ? align16(sizeof(T) * N * N * N * N) : 0) +
         align16(cg_tile_values<T, N>(TY, TX) * sizeof(T) > pc_line_bytes<T, N>(kind, Lmax, pow2)
                     ? cg_tile_values<T, N>(TY, TX) * sizeof(T)
                     : pc_line_bytes<T, N>(kind, Lmax, pow2));
}

// Lays out the solve context over dynamic shared memory starting at base (bytes).
template <typename T, int N, typename TB = T>
__device__ __forceinline__ void init_ctx(SolveCtx<T>& X, unsigned char* base, const Geom& G, const TB* Bt_global,
                                         bool pc, int Lmax) {
  constexpr int NN = N * N;
  unsigned char* p = base;
  if (pc) {
    TB* Bs = reinterpret_cast<TB*>(p);  // Bt in the preconditioner's precision TB (<= T)
    for (int i = threadIdx.x; i < NN * NN; i += blockDim.x) Bs[i] = Bt_global[i];
    X.Bs = reinterpret_cast<const T*>(Bs);
    p += align16(sizeof(T) * NN * NN);
  } else {
    X.Bs = nullptr;
  }
  const int boxc = (G.TY + 2) * (G.TX + 2);
  X.sU = reinterpret_cast<T*>(p);
  X.tXR = X.sU + boxc * (NN + 1);
  X.tXL = X.tXR + boxc * N;
  X.tYR = X.tXL + boxc * N;
  X.tYL = X.tYR + boxc * N;
  X.line0 = reinterpret_cast<Cplx<T>*>(p);
  X.line1 = X.line0 + Lmax;
  X.cluster = 0;
  X.kdf = nullptr;
  X.wU = X.wXR = X.wXL = X.wYR = X.wYL = nullptr;
  __syncthreads();
}

// The whole Poisson solve on the (virtual) grid of X (context laid out by init_ctx).
template <typename T, int N, typename TP = T>
__device__ __forceinline__ void cg_solve(const Ops2D<T, N>& C, const Geom& G, const CgArgs<T, TP>& A,
                                         SolveCtx<T>& X) {
  constexpr int NN = N * N;
  const bool pc = A.precond != kPrecondJacobi;
  X.sync = A.sync;
  X.part = A.part;
  X.phase = 0;
  X.tbase = read_ticket<T>(A.sync);  // before the first barrier: no block has drawn yet
  const int ntiles = G.tilesX * G.tilesY;
  const size_t ndof = (size_t)G.Nx * G.Ny * NN;
  const size_t stride = (size_t)X.vsize * blockDim.x;
  int flags = 0, it = 0;
  T rr = T(0), rhob = T(0), rz = T(0);

  // P0: W-mean of omega, in two passes (the second removes the rounding left by the first,
  // so that b carries no rounding-sized component along the kernel of A).
  T wbar = T(0);
  if (A.rhs == nullptr && !A.keep_mean) {
    for (int pass = 0; pass < 2; ++pass) {
      T s = T(0);
      strided_pass<4>((size_t)X.vrank * blockDim.x + threadIdx.x, ndof, stride,
                      [&](size_t i) { return T(A.omega[i]); },
                      [&](size_t i, T v) { s = fma(C.wq[i % NN], v - wbar, s); });
      T m = T(0);
      if (!reduce_all(X, s, m)) {
        flags |= kFlagTimeout;
        goto finish;
      }
      wbar += m / T(A.sumW);
    }
  }
  // P1: y0, b, r0 = b - Ahat y0, rr0 = r0.r0, rhob = b.b.
  if (A.axa) {  // Ahat y0 from the recycled products: a pointwise pass
    T rrb = T(0), bbb = T(0);
    const RhsSource<T> src{A.omega, A.rhs, wbar};
    for (size_t g = (size_t)X.vrank * blockDim.x + threadIdx.x; g < ndof; g += stride) {
      const int k = int(g % NN);
      T y0 = T(0), ax = T(0);
      if (A.xa) {
        y0 = T(A.ca) * T(A.xa[g]);
        ax = T(A.ca) * __ldcg(A.axa + g);
      }
      if (A.xb) {
        y0 = fma(T(A.cb), T(A.xb[g]), y0);
        ax = fma(T(A.cb), __ldcg(A.axb + g), ax);
      }
      __stcg(A.v.y + g, y0);
      const T b = rhs_at<T, N>(C, src, g, k);
      const T r = b - ax;
      __stcg(A.v.r + g, r);
      rrb = fma(r, r, rrb);
      bbb = fma(b, b, bbb);
    }
    if (!reduce_all2(X, rrb, bbb, rr, rhob)) {
      flags |= kFlagTimeout;
      goto finish;
    }
  } else {
    T rrb = T(0), bbb = T(0);
    for (int t = X.vrank; t < ntiles; t += X.vsize) {
      cg_tile_apply<T, N>(
          C, G, t, X,
          [&](size_t g, int k, bool interior) {
            double v = 0.0;
            if (A.xa) v = A.ca * A.xa[g];
            if (A.xb) v = fma(A.cb, A.xb[g], v);
            T tv = A.x_unscaled ? T(v) * C.sw[k] : T(v);
            if (interior) __stcg(A.v.y + g, tv);
            return tv;
          },
          [&](size_t g, int k, T, T qv) {
            const T b = rhs_at<T, N>(C, RhsSource<T>{A.omega, A.rhs, wbar}, g, k);
            const T r = b - qv;
            __stcg(A.v.r + g, r);
            rrb = fma(r, r, rrb);
            bbb = fma(b, b, bbb);
          });
    }
    if (!reduce_all2(X, rrb, bbb, rr, rhob)) {
      flags |= kFlagTimeout;
      goto finish;
    }
  }
  if (rhob == T(0)) {
    for (size_t i = (size_t)X.vrank * blockDim.x + threadIdx.x; i < ndof; i += stride) __stcg(A.v.y + i, T(0));
    rr = T(0);
  } else {
    if (pc && !pc_apply<T, N, TP>(C, G, A.pc, A.v.r, X, rz)) {
      flags |= kFlagTimeout;
      goto finish;
    }
    it = cg_iterate<T, N, TP>(C, G, A.v, pc ? &A.pc : nullptr, RhsSource<T>{A.omega, A.rhs, wbar}, X, rr, rz, rhob,
                              A.tol2, A.maxit, A.fixed_iters, flags, kMaxRestarts, A.floor2, A.ay);
    if (pc && !(flags & kFlagTimeout) && !project_mean<T, N>(C, G, A.v.y, A.sumW, X)) flags |= kFlagTimeout;
  }
finish:
  if (A.psi_out && !(flags & kFlagTimeout)) {
    strided_pass<4>((size_t)X.vrank * blockDim.x + threadIdx.x, ndof, stride,
                    [&](size_t i) { return __ldcg(A.v.y + i); },
                    [&](size_t i, T v) { A.psi_out[i] = double(v * C.isw[i % NN]); });
  }
  if (X.vrank == 0 && threadIdx.x == 0) {
    SolveStatus* st = A.status;
    st->total_iters += it;
    st->last_iters = it;
    st->max_iters = max(st->max_iters, it);
    st->last_flags = flags;
    st->flags |= flags;
    st->nsolves += 1;
    st->last_sweeps = 0;
    st->last_rho = double(rr);
    st->last_rhob = double(rhob);
  }
}

// MinB: the blocks per SM the register budget is sized for.  The solves with the spectral
// preconditioner are launched with MinB = 2 (up to 128 registers a thread: its V transforms
// keep n complex values per row in registers, and its line buffers allow two blocks per SM on
// large grids anyway).
template <typename T, int N, typename TP = T, int MinB = (N == 5 ? 4 : 3)>
__global__ void __launch_bounds__(kThreads, MinB) cg_kernel(const __grid_constant__ Ops2D<T, N> C, const Geom G,
                                                        const __grid_constant__ CgArgs<T, TP> A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ T red[32];
  __shared__ T bcast;
  __shared__ int s_flag;
  const Ops2D<T, N>& Cs = stage_table(C, smem_raw);
  SolveCtx<T> X;
  init_ctx<T, N, TP>(X, smem_raw + table_bytes<Ops2D<T, N>>(), G, A.pc.Bt, A.precond == 1, max(G.Nx, G.Ny));
  X.red = red;
  X.bcast = &bcast;
  X.s_flag = &s_flag;
  X.vrank = blockIdx.x;
  X.vsize = gridDim.x;
  X.cluster = A.cluster;
  cg_solve<T, N, TP>(Cs, G, A, X);
}

// =========================================================================================
// Mixed precision Poisson solve (iterative refinement, all on the device):
//   y  <- y0;  r = b - Ahat y  in float64
//   while r.r > tol^2 b.b:  solve Ahat e = r in float32 by CG from e = 0 to the relative
//                           tolerance tol_in;  y += e (float64);  r = b - Ahat y (float64)
// The float64 residual is the true residual of the float64 iterate, so the outer stopping
// rule needs no further check.
// =========================================================================================
struct MixedArgs {
  const double* omega;
  const double* xa;
  const double* xb;
  double ca, cb;
  int x_unscaled;
  const double* axa;   // recycled operator products, as in CgArgs
  const double* axb;
  double* ay;
  double* y;           // float64 solution (scaled space)
  double* psi_out;     // if non-null: psi = y / sqrt(W) at the end
  float* rf;           // float32 copy of the float64 residual (inner right-hand side)
  CgVectors<float> v;  // inner solve: y = e, r, p0, p1, q
  int precond;         // kPrecondJacobi, kPrecondTwoLevel or kPrecondSpectral (inner float32 solve)
  PrecondArgs<float> pc;
  double* partd;       // 6 * gridDim.x
  float* partf;        // 6 * gridDim.x
  SyncState* sync;
  SolveStatus* status;
  double tol2, tol_in2;
  double floor2;       // the float64 rounding floor per unit y.y (see CgArgs::floor2)
  int max_sweeps, maxit_in;
  double sumW;
  int cluster;         // launched as one thread-block cluster (cluster barriers)
  // the inner solve's operator apply (see solve_apply): 0 float32, 1 double-float, 2 float32
  // until a refinement sweep after the second reduces the residual by less than a factor 100
  // (too inexact on this problem's smoothest modes), double-float from then on
  int precise_apply;
  int keep_mean;       // homogeneous Dirichlet: b = sqrt(W) omega (no mean removed)
};

// The operator tables a mixed solve stages in shared memory: float64 (residuals), float32
// (inner solve) and the double-float CG operator (compensated apply).
template <int N>
__host__ __device__ constexpr size_t mixed_ops_bytes() {
  return table_bytes<Ops2D<double, N>>() + table_bytes<Ops2D<float, N>>() + table_bytes<OpsK<df, N>>();
}

template <int N>
__host__ __device__ constexpr size_t mixed_smem_bytes(int TY, int TX, int Lmax, int kind, bool pow2) {
  return (kind == kPrecondTwoLevel ? align16(sizeof(float) * N * N * N * N) : 0) +
         align16(cg_tile_values<double, N>(TY, TX) * sizeof(double) > pc_line_bytes<float, N>(kind, Lmax, pow2)
                     ? cg_tile_values<double, N>(TY, TX) * sizeof(double)
                     : pc_line_bytes<float, N>(kind, Lmax, pow2));
}

// One float64 residual pass: r = b - Ahat y (y staged with halo; pass 0: y = y0), rf =
// float(r), inner residual = rf, e = 0.  Accumulates this block's r.r and b.b.
template <int N>
__device__ __forceinline__ void mixed_residual(const Ops2D<double, N>& Cd, const Geom& G, const MixedArgs& A,
                                               double wbar, bool from_x0, SolveCtx<double>& X, double& rr,
                                               double& bb, double& yy) {
  constexpr int NN = N * N;
  if (from_x0 && A.axa) {  // Ahat y0 from the recycled products: a pointwise pass
    const size_t ndof = (size_t)G.Nx * G.Ny * NN;
    for (size_t g = (size_t)X.vrank * blockDim.x + threadIdx.x; g < ndof; g += (size_t)X.vsize * blockDim.x) {
      const int k = int(g % NN);
      double y0 = 0.0, ax = 0.0;
      if (A.xa) {
        y0 = A.ca * A.xa[g];
        ax = A.ca * __ldcg(A.axa + g);
      }
      if (A.xb) {
        y0 = fma(A.cb, A.xb[g], y0);
        ax = fma(A.cb, __ldcg(A.axb + g), ax);
      }
      __stcg(A.y + g, y0);
      if (A.ay) __stcg(A.ay + g, ax);
      const double b = Cd.sw[k] * (A.omega[g] - wbar);
      const double r = b - ax;
      const float r32 = float(r);
      __stcg(A.rf + g, r32);
      __stcg(A.v.r + g, r32);
      __stcg(A.v.y + g, 0.0f);
      rr = fma(r, r, rr);
      bb = fma(b, b, bb);
      yy = fma(y0, y0, yy);
    }
    return;
  }
  const int ntiles = G.tilesX * G.tilesY;
  for (int t = X.vrank; t < ntiles; t += X.vsize) {
    cg_tile_apply<double, N>(
        Cd, G, t, X,
        [&](size_t g, int k, bool interior) {
          if (!from_x0) return __ldcg(A.y + g);
          double v = 0.0;
          if (A.xa) v = A.ca * A.xa[g];
          if (A.xb) v = fma(A.cb, A.xb[g], v);
          if (A.x_unscaled) v *= Cd.sw[k];
          if (interior) __stcg(A.y + g, v);
          return v;
        },
        [&](size_t g, int k, double yv, double qv) {
          const double b = Cd.sw[k] * (A.omega[g] - wbar);
          const double r = b - qv;
          if (A.ay) __stcg(A.ay + g, qv);
          const float r32 = float(r);
          __stcg(A.rf + g, r32);
          __stcg(A.v.r + g, r32);
          __stcg(A.v.y + g, 0.0f);
          rr = fma(r, r, rr);
          bb = fma(b, b, bb);
          yy = fma(yv, yv, yy);
        });
  }
}

// The whole mixed-precision solve on the (virtual) grid of Xf / Xd (float context with the
// staged block matrix, double context over the same region; see mixed_cg_kernel).
template <int N>
__device__ __forceinline__ void mixed_solve(const Ops2D<double, N>& Cd, const Ops2D<float, N>& Cf,
                                            const OpsK<df, N>& Ck, const Geom& G, const MixedArgs& A,
                                            SolveCtx<float>& Xf, SolveCtx<double>& Xd) {
  constexpr int NN = N * N;
  const bool pc = A.precond != kPrecondJacobi;
  // the double-float apply stages its tiles in the float64 buffers
  Xf.wU = reinterpret_cast<df*>(Xd.sU);
  Xf.wXR = reinterpret_cast<df*>(Xd.tXR);
  Xf.wXL = reinterpret_cast<df*>(Xd.tXL);
  Xf.wYR = reinterpret_cast<df*>(Xd.tYR);
  Xf.wYL = reinterpret_cast<df*>(Xd.tYL);
  Xf.kdf = A.precise_apply == 1 ? &Ck : nullptr;
  Xf.sync = A.sync;
  Xf.part = A.partf;
  Xf.phase = 0;
  Xd.sync = A.sync;
  Xd.part = A.partd;
  Xd.phase = 0;
  Xf.tbase = Xd.tbase = read_ticket<float>(A.sync);  // before the first barrier
  const size_t ndof = (size_t)G.Nx * G.Ny * NN;
  const size_t stride = (size_t)Xd.vsize * blockDim.x;
  int flags = 0, sweeps = 0;
  long long inner = 0;
  double rr = 0.0, bb = 0.0, wbar = 0.0, rr_prev = -1.0;
  for (int mp = 0; mp < (A.keep_mean ? 0 : 2); ++mp) {  // two-pass W-mean, as in cg_kernel
    double s = 0.0;
    strided_pass<4>((size_t)Xd.vrank * blockDim.x + threadIdx.x, ndof, stride,
                    [&](size_t i) { return A.omega[i]; },
                    [&](size_t i, double v) { s = fma(Cd.wq[i % NN], v - wbar, s); });
    double m = 0.0;
    if (!reduce_all(Xd, s, m)) {
      flags |= kFlagTimeout;
      goto finish;
    }
    wbar += m / A.sumW;
  }
  for (int pass = 0;; ++pass) {
    // float64 residual of the current iterate (pass 0: of the initial guess)
    double yy = 0.0;
    {
      double r2 = 0.0, b2 = 0.0, y2 = 0.0;
      mixed_residual<N>(Cd, G, A, wbar, pass == 0, Xd, r2, b2, y2);
      if (!reduce_all3(Xd, r2, b2, y2, rr, bb, yy)) {
        flags |= kFlagTimeout;
        goto finish;
      }
    }
    if (bb == 0.0) {
      for (size_t i = (size_t)Xd.vrank * blockDim.x + threadIdx.x; i < ndof; i += stride) __stcg(A.y + i, 0.0);
      rr = 0.0;
      break;
    }
    if (Xd.vrank == 0 && threadIdx.x == 0 && pass < kRefineHistory) {
      A.status->hist_rr[pass] = rr / bb;
      A.status->hist_len = pass + 1;
    }
    if (rr <= A.tol2 * bb) break;
    // stagnation at the float64 rounding floor of y (see CgArgs::floor2): below it, and less
    // than a factor 4 below the previous sweep's residual
    if (rr <= A.floor2 * yy && rr_prev >= 0.0 && rr > 0.25 * rr_prev) break;
    // adaptive apply: a sweep after the second that gained less than a factor 100 in the
    // residual norm (1e-4 in r.r) switches the inner solves to the double-float apply (the
    // first sweep from a poor guess is limited by the float32 rounding of its large correction
    // instead)
    if (A.precise_apply == 2 && !Xf.kdf && pass >= 2 && rr > 1e-4 * rr_prev) Xf.kdf = &Ck;
    rr_prev = rr;
    if (sweeps >= A.max_sweeps) {
      flags |= kFlagNoconv;
      break;
    }
    // float32 inner (P)CG from e = 0 on the residual equation, to the relative tolerance
    // tol_in -- or to what is left to reach the outer tolerance (with a factor 1/2 of
    // margin), if that is looser: the last sweep then does only the iterations it needs
    const double tol_eff2 = fmax(A.tol_in2, 0.25 * A.tol2 * bb / rr);
    float rho_in = float(rr);
    const float rhob_in = rho_in;
    float rz_in = rho_in;
    if (pc && !pc_apply<float, N>(Cf, G, A.pc, A.v.r, Xf, rz_in)) {
      flags |= kFlagTimeout;
      goto finish;
    }
    int fin = 0;
    const int it_in = cg_iterate<float, N>(Cf, G, A.v, pc ? &A.pc : nullptr, RhsSource<float>{nullptr, A.rf, 0.0f},
                                           Xf, rho_in, rz_in, rhob_in, tol_eff2, A.maxit_in, 0, fin, 0);
    inner += it_in;
    if (Xd.vrank == 0 && threadIdx.x == 0 && pass < kRefineHistory) A.status->hist_it[pass] = it_in;
    if (fin & kFlagTimeout) {
      flags |= kFlagTimeout;
      goto finish;
    }
    // y += e
    struct Ye {
      double y;
      float e;
    };
    strided_pass<4>((size_t)Xd.vrank * blockDim.x + threadIdx.x, ndof, stride,
                    [&](size_t i) { return Ye{__ldcg(A.y + i), __ldcg(A.v.y + i)}; },
                    [&](size_t i, const Ye& v) { __stcg(A.y + i, v.y + double(v.e)); });
    if (!solve_barrier(Xd)) {
      flags |= kFlagTimeout;
      goto finish;
    }
    ++sweeps;
  }
  if (pc && !(flags & kFlagTimeout) && !project_mean<double, N>(Cd, G, A.y, A.sumW, Xd)) flags |= kFlagTimeout;
finish:
  if (A.psi_out && !(flags & kFlagTimeout)) {
    strided_pass<4>((size_t)Xd.vrank * blockDim.x + threadIdx.x, ndof, stride,
                    [&](size_t i) { return __ldcg(A.y + i); },
                    [&](size_t i, double v) { A.psi_out[i] = v * Cd.isw[i % NN]; });
  }
  if (Xd.vrank == 0 && threadIdx.x == 0) {
    SolveStatus* st = A.status;
    const int it = int(inner);
    st->total_iters += it;
    st->last_iters = it;
    st->max_iters = max(st->max_iters, it);
    st->last_flags = flags;
    st->flags |= flags;
    st->nsolves += 1;
    st->last_sweeps = sweeps;
    st->last_rho = rr;
    st->last_rhob = bb;
  }
}

template <int N, int MinB = 4>
__global__ void __launch_bounds__(kThreads, MinB) mixed_cg_kernel(const __grid_constant__ Ops2D<double, N> Cd,
                                                           const __grid_constant__ Ops2D<float, N> Cf,
                                                           const __grid_constant__ OpsK<df, N> Ck, const Geom G,
                                                           const __grid_constant__ MixedArgs A) {
  constexpr int NN = N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ double bcd;
  __shared__ float redf[32];
  __shared__ float bcf;
  __shared__ int s_flag;
  const bool pc = A.precond == kPrecondTwoLevel;  // the cell blocks are staged
  const int Lmax = max(G.Nx, G.Ny);
  const Ops2D<double, N>& Cds = stage_table(Cd, smem_raw);
  const Ops2D<float, N>& Cfs = stage_table(Cf, smem_raw + table_bytes<Ops2D<double, N>>());
  const OpsK<df, N>& Cks =
      stage_table(Ck, smem_raw + table_bytes<Ops2D<double, N>>() + table_bytes<Ops2D<float, N>>());
  unsigned char* smem = smem_raw + mixed_ops_bytes<N>();
  SolveCtx<float> Xf;
  init_ctx<float, N>(Xf, smem, G, A.pc.Bt, pc, Lmax);
  Xf.red = redf;
  Xf.bcast = &bcf;
  Xf.s_flag = &s_flag;
  Xf.vrank = blockIdx.x;
  Xf.vsize = gridDim.x;
  SolveCtx<double> Xd;
  init_ctx<double, N>(Xd, smem + (pc ? align16(sizeof(float) * NN * NN) : 0), G, (const double*)nullptr, false, Lmax);
  Xd.red = redd;
  Xd.bcast = &bcd;
  Xd.s_flag = &s_flag;
  Xd.vrank = blockIdx.x;
  Xd.vsize = gridDim.x;
  Xf.cluster = Xd.cluster = A.cluster;
  mixed_solve<N>(Cds, Cfs, Cks, G, A, Xf, Xd);
}

// =========================================================================================
// Batched persistent step: many independent simulations (different grids, n, viscosities)
// advance in one cooperative launch.  The blocks are split into groups; each group is a
// virtual grid (its own barrier, block ranks and partial sums) that runs whole AB3 steps --
// the RHS tile pass, the Poisson solve, the rotation of the state rings -- for the
// simulations queued on it, one after the other.  Groups run concurrently.
// =========================================================================================
struct BatchSim {
  int n, precision, precond;       // precision: 0 float64, 1 mixed (double-float RHS), 2 mixed (float64 RHS)
  int precise_apply;               // mixed: the inner solve applies Ahat in double-float
  int keep_mean;                   // homogeneous Dirichlet grid: no mean removed from omega
  Geom Gr, Gc;                     // tiles of the RHS and of the solve
  const void* ops_d;               // device copy of Ops2D<double, n>
  const void* ops_f;               // device copy of Ops2D<float, n>
  const void* ops_df;              // device copy of Ops2D<df, n> (double-float RHS)
  const void* ops_k;               // device copy of OpsK<df, n> (double-float CG operator)
  double* omega[2];
  double* psi[3];                  // sqrt(W) psi
  double* apsi[3];                 // Ahat psi of each slot, valid where apsi_ok (see dg_sim)
  int apsi_ok[3];
  void* R[4];                      // right-hand-side history (float64)
  int oc, p0, p1, p2, r1, r2, r3, rfree;  // ring indices, advanced by the kernel
  long long step;
  long long limit;                 // no batched step once step == limit (0: no limit)
  double D, dt, tol2, tol_in2, floor2;
  int maxit, max_sweeps, fixed_iters;
  double sumW;
  // float64 solve
  double *r, *p0v, *p1v, *q, *part;
  // mixed solve
  float *rf, *fr, *fe, *fp0, *fp1, *fq, *partf;
  SolveStatus* status;
  PrecondArgs<double> pc;
  PrecondArgs<float> pcf;
};

struct BatchGroup {
  int first_block, nblocks;  // blocks [first_block, first_block + nblocks)
  int first, count;          // simulations order[first .. first + count)
  SyncState* sync;
};

struct BatchArgs {
  BatchSim* sims;
  const int* order;
  const BatchGroup* groups;
  int ngroups;
  int nsteps;
  int* error;                // first error flag of any group
};

template <typename T, int N>
__device__ __noinline__ void batch_rhs(const BatchSim& S, const Ops2D<T, N>& C, int oc, int p0, int r1, int r2,
                                          int rfree, int vrank, int vsize, unsigned char* smem) {
  RhsArgs<T> A{};
  A.psi = S.psi[p0];
  A.omega_in = S.omega[oc];
  A.omega_base = S.omega[oc];
  A.omega_out = S.omega[oc ^ 1];
  A.R_out = static_cast<hist_t<T>*>(S.R[rfree]);
  A.hist[0] = static_cast<const hist_t<T>*>(S.R[r1]);
  A.hist[1] = static_cast<const hist_t<T>*>(S.R[r2]);
  A.c_new = 23.0 / 12.0;
  A.c_hist[0] = -16.0 / 12.0;
  A.c_hist[1] = 5.0 / 12.0;
  A.nhist = 2;
  A.dt = S.dt;
  A.visc = S.D;
  A.psi_scaled = 1;
  const int nt = S.Gr.tilesX * S.Gr.tilesY;
  for (int t = vrank; t < nt; t += vsize) rhs_tile<T, N>(C, S.Gr, A, t, smem);
}

// One AB3 step of simulation S on a group.  Returns false after a barrier timeout.
// Shared-memory tables of a batched step: the float64 operators (the double-float RHS
// operators during a DG_MIXED member's RHS pass: same size), float32, double-float CG operator.
template <int N>
__host__ __device__ constexpr size_t batch_ops_bytes() {
  static_assert(sizeof(Ops2D<df, N>) == sizeof(Ops2D<double, N>), "table sizes");
  return table_bytes<Ops2D<double, N>>() + table_bytes<Ops2D<float, N>>() + table_bytes<OpsK<df, N>>();
}

template <int N>
__device__ __noinline__ bool batch_step(BatchSim* Sp, const BatchGroup& grp, int vrank, unsigned char* smem_all,
                                           double* redd, double* bcd, float* redf, float* bcf, int* s_flag) {
  constexpr int NN = N * N;
  const BatchSim& S = *Sp;
  // a simulation that has reached its step limit sits the step out (every block of the
  // group reads the same step index: it was written before the group's last barrier)
  if (S.limit > 0 && __ldcg(&Sp->step) >= S.limit) return true;
  const int oc = __ldcg(&Sp->oc), p0 = __ldcg(&Sp->p0), p1 = __ldcg(&Sp->p1), p2 = __ldcg(&Sp->p2);
  const int r1 = __ldcg(&Sp->r1), r2 = __ldcg(&Sp->r2), r3 = __ldcg(&Sp->r3), rfree = __ldcg(&Sp->rfree);
  // this simulation's operator tables, staged in shared memory (the previous step's last
  // barrier has synchronised the block)
  unsigned char* smem = smem_all + batch_ops_bytes<N>();
  if (S.precision == 1) {
    const Ops2D<df, N>& Cr = stage_table(*static_cast<const Ops2D<df, N>*>(S.ops_df), smem_all);
    batch_rhs<df, N>(S, Cr, oc, p0, r1, r2, rfree, vrank, grp.nblocks, smem);
  } else {
    const Ops2D<double, N>& Cr = stage_table(*static_cast<const Ops2D<double, N>*>(S.ops_d), smem_all);
    batch_rhs<double, N>(S, Cr, oc, p0, r1, r2, rfree, vrank, grp.nblocks, smem);
  }
  if (!grid_barrier(grp.sync, s_flag, grp.nblocks)) return false;
  // the solve's tables (the barrier has synchronised the block: the RHS table is no longer read)
  const Ops2D<double, N>& Cd = stage_table(*static_cast<const Ops2D<double, N>*>(S.ops_d), smem_all);
  const Ops2D<float, N>& Cf =
      stage_table(*static_cast<const Ops2D<float, N>*>(S.ops_f), smem_all + table_bytes<Ops2D<double, N>>());
  const OpsK<df, N>& Ck = stage_table(*static_cast<const OpsK<df, N>*>(S.ops_k),
                                      smem_all + table_bytes<Ops2D<double, N>>() + table_bytes<Ops2D<float, N>>());
  const bool pc = S.precond == kPrecondTwoLevel;  // the cell blocks are staged
  const int Lmax = max(S.Gc.Nx, S.Gc.Ny);
  // the initial residual from the kept operator products (as in the single-simulation stepper)
  const bool rec = S.fixed_iters == 0 && __ldcg(&Sp->apsi_ok[p0]) && __ldcg(&Sp->apsi_ok[p1]);
  if (S.precision == 0) {
    CgArgs<double> A{};
    A.omega = S.omega[oc ^ 1];
    A.xa = S.psi[p0];
    A.xb = S.psi[p1];
    A.ca = 2.0;
    A.cb = -1.0;
    if (rec) {
      A.axa = S.apsi[p0];
      A.axb = S.apsi[p1];
    }
    if (S.fixed_iters == 0) A.ay = S.apsi[p2];
    A.v = CgVectors<double>{S.psi[p2], S.r, S.p0v, S.p1v, S.q};
    A.precond = S.precond;
    A.pc = S.pc;
    A.part = S.part;
    A.sync = grp.sync;
    A.status = S.status;
    A.tol2 = S.tol2;
    A.floor2 = S.floor2;
    A.keep_mean = S.keep_mean;
    A.maxit = S.fixed_iters > 0 ? max(S.maxit, S.fixed_iters) : S.maxit;
    A.fixed_iters = S.fixed_iters;
    A.sumW = S.sumW;
    SolveCtx<double> X;
    init_ctx<double, N>(X, smem, S.Gc, S.pc.Bt, pc, Lmax);
    X.red = redd;
    X.bcast = bcd;
    X.s_flag = s_flag;
    X.vrank = vrank;
    X.vsize = grp.nblocks;
    cg_solve<double, N>(Cd, S.Gc, A, X);
  } else {
    MixedArgs A{};
    A.omega = S.omega[oc ^ 1];
    A.xa = S.psi[p0];
    A.xb = S.psi[p1];
    A.ca = 2.0;
    A.cb = -1.0;
    if (rec) {
      A.axa = S.apsi[p0];
      A.axb = S.apsi[p1];
    }
    if (S.fixed_iters == 0) A.ay = S.apsi[p2];
    A.y = S.psi[p2];
    A.rf = S.rf;
    A.v = CgVectors<float>{S.fe, S.fr, S.fp0, S.fp1, S.fq};
    A.precond = S.precond;
    A.pc = S.pcf;
    A.partd = S.part;
    A.partf = S.partf;
    A.sync = grp.sync;
    A.status = S.status;
    A.tol2 = S.tol2;
    A.floor2 = S.floor2;
    A.keep_mean = S.keep_mean;
    A.tol_in2 = S.tol_in2;
    A.max_sweeps = S.max_sweeps;
    A.maxit_in = S.maxit;
    A.sumW = S.sumW;
    A.precise_apply = S.precise_apply;
    SolveCtx<float> Xf;
    init_ctx<float, N>(Xf, smem, S.Gc, S.pcf.Bt, pc, Lmax);
    Xf.red = redf;
    Xf.bcast = bcf;
    Xf.s_flag = s_flag;
    Xf.vrank = vrank;
    Xf.vsize = grp.nblocks;
    SolveCtx<double> Xd;
    init_ctx<double, N>(Xd, smem + (pc ? align16(sizeof(float) * NN * NN) : 0), S.Gc, (const double*)nullptr, false, Lmax);
    Xd.red = redd;
    Xd.bcast = bcd;
    Xd.s_flag = s_flag;
    Xd.vrank = vrank;
    Xd.vsize = grp.nblocks;
    mixed_solve<N>(Cd, Cf, Ck, S.Gc, A, Xf, Xd);
  }
  // every block has finished the solve before the rings move
  if (!grid_barrier(grp.sync, s_flag, grp.nblocks)) return false;
  if (vrank == 0 && threadIdx.x == 0) {
    Sp->apsi_ok[p2] = S.fixed_iters == 0 ? 1 : 0;
    Sp->oc = oc ^ 1;
    Sp->p0 = p2;
    Sp->p1 = p0;
    Sp->p2 = p1;
    Sp->r1 = rfree;
    Sp->r2 = r1;
    Sp->r3 = r2;
    Sp->rfree = r3;
    Sp->step = S.step + 1;
    __threadfence();
  }
  return grid_barrier(grp.sync, s_flag, grp.nblocks);
}



// =========================================================================================
// Invariants: partial sums of W omega, W psi omega, W omega^2 per block, then one block
// adds the partials in a fixed order.
// =========================================================================================
template <int N>
struct NodeWeights {
  double w[N * N];    // W_ab
  double sw[N * N];   // sqrt(W_ab)
  double isw[N * N];  // 1 / sqrt(W_ab)
};

template <int N>
__global__ void __launch_bounds__(kThreads) invariants_partial_kernel(const __grid_constant__ NodeWeights<N> W,
                                                                     const double* __restrict__ psi,
                                                                     const double* __restrict__ omega,
                                                                     size_t ndof, int psi_scaled,
                                                                     double* __restrict__ part) {
  constexpr int NN = N * N;
  __shared__ double red[32];
  double v = 0.0, e = 0.0, o = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += (size_t)gridDim.x * blockDim.x) {
    const int k = int(i % NN);
    const double w = omega[i];
    const double p = psi_scaled ? psi[i] * W.isw[k] : psi[i];
    const double ww = W.w[k] * w;
    v += ww;
    e = fma(ww, p, e);
    o = fma(ww, w, o);
  }
  v = block_sum(v, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x] = v;
  e = block_sum(e, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 1] = e;
  o = block_sum(o, red);
  if (threadIdx.x == 0) part[3 * blockIdx.x + 2] = o;
}


// ---- small elementwise kernels ----------------------------------------------------------

// y[i] = x[i] * s[i % NN]   (psi <-> sqrt(W) psi)
template <int N>
__global__ void scale_nodes_kernel(const __grid_constant__ NodeWeights<N> W, const double* __restrict__ x,
                                   double* __restrict__ y, size_t ndof, int inverse) {
  constexpr int NN = N * N;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndof; i += (size_t)gridDim.x * blockDim.x) {
    const int k = int(i % NN);
    y[i] = x[i] * (inverse ? W.isw[k] : W.sw[k]);
  }
}


}  // namespace dgk
