// Internal host-side declarations shared by the translation units of libdgk: error
// reporting, the handle structs (dg_grid, dg_sim and their device workspace), tile choices,
// small helpers, and the per-n kernel launchers.  The launchers are defined in
// dg_launch.cuh and instantiated once per n in dg_inst_n<N>.cu, so that the kernels of each
// n compile in a translation unit of their own (in parallel).
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/dg.h"
#include "dg_kernels.cuh"
#include "dg_tables.h"

namespace dgk {

// Message of the last error on this thread (dg_last_error); defined in dg_capi.cu.
extern thread_local char g_err[512];

inline int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(e_ == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA, \
                                       "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

inline cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

// Host copies of the device operator tables for one n, in float64 and float32.
struct OpsHost {
  alignas(16) unsigned char d[sizeof(Ops2D<double, kMaxN>)];
  alignas(16) unsigned char f[sizeof(Ops2D<float, kMaxN>)];
  alignas(16) unsigned char x[sizeof(Ops2D<df, kMaxN>)];  // double-float (RHS of DG_MIXED)
  alignas(16) unsigned char k[sizeof(OpsK<df, kMaxN>)];   // double-float CG operator
};

template <int N>
NodeWeights<N> make_weights(const RefTables& t, double hx, double hy) {
  NodeWeights<N> W;
  for (int a = 0; a < N; ++a)
    for (int b = 0; b < N; ++b) {
      const double w = (hy * 0.5 * t.w[a]) * (hx * 0.5 * t.w[b]);
      W.w[a * N + b] = w;
      W.sw[a * N + b] = std::sqrt(w);
      W.isw[a * N + b] = 1.0 / std::sqrt(w);
    }
  return W;
}

// Built-in tiles (cells per block, TY x TX) for the RHS kernel and the CG kernel.
inline void default_tiles(int n, int& rty, int& rtx, int& cty, int& ctx) {
  static const int R[6][2] = {{0, 0}, {16, 16}, {8, 16}, {8, 8}, {4, 8}, {4, 8}};
  static const int Cg[6][2] = {{0, 0}, {16, 16}, {16, 16}, {8, 16}, {8, 8}, {8, 8}};
  rty = R[n][0];
  rtx = R[n][1];
  cty = Cg[n][0];
  ctx = Cg[n][1];
}

// Small grids: halve the larger tile side until the grid has at least one tile per SM (or
// the tile is down to 4 cells), so that the few cells are spread over many blocks -- the
// solves' phases are then short chains of work rather than long loops in a few blocks.
inline void fit_tile(int Nx, int Ny, int sms, int& ty, int& tx) {
  auto tiles = [&]() { return (long long)((Nx + tx - 1) / tx) * ((Ny + ty - 1) / ty); };
  while (tiles() < sms && ty * tx > 4) {
    if (tx >= ty && tx > 1)
      tx /= 2;
    else if (ty > 1)
      ty /= 2;
    else
      break;
  }
}

inline void choose_tiles(int n, int Nx, int Ny, int sms, int& rty, int& rtx, int& cty, int& ctx) {
  default_tiles(n, rty, rtx, cty, ctx);
  // a single simulation's RHS kernel at n = 5 is faster on 8 x 8 tiles (1024^2 cells:
  // 5.5 against 6.6 ms per bracket), whose ~200 KB of shared memory a batch, sizing its
  // kernel for every member, would pay in resident blocks: batches keep 4 x 8
  if (n == 5) rty = 8;
  fit_tile(Nx, Ny, sms, rty, rtx);
  fit_tile(Nx, Ny, sms, cty, ctx);
}

}  // namespace dgk

using namespace dgk;

// ---------------------------------------------------------------------------------------
// Handles
// ---------------------------------------------------------------------------------------

struct Workspace {
  size_t ndof = 0;
  int grid_cap = 0;  // capacity of the partials (blocks)
  double *r = nullptr, *p0 = nullptr, *p1 = nullptr, *q = nullptr, *y = nullptr;
  double* part = nullptr;  // 6 * grid_cap
  // float32 inner-solve vectors of the mixed precision path
  float *rf = nullptr, *fr = nullptr, *fe = nullptr, *fp0 = nullptr, *fp1 = nullptr, *fq = nullptr;
  float* partf = nullptr;
  // two-level preconditioner work arrays (float64 and, for the mixed path, float32)
  double *pz = nullptr, *prc = nullptr, *puc = nullptr;
  Cplx<double>* pC = nullptr;
  float *pzf = nullptr, *prcf = nullptr, *pucf = nullptr;
  Cplx<float>* pCf = nullptr;
  // spectrum of the spectral preconditioner, (Nx/2 + 1) x Ny x n x n (float64 and float32)
  Cplx<double>* pS = nullptr;
  Cplx<float>* pSf = nullptr;
  SyncState* sync = nullptr;
  SolveStatus* status = nullptr;
  double* inv_part = nullptr;  // 3 * kInvBlocks
  double* inv_out = nullptr;   // 3
  double* host_out = nullptr;  // pinned 3
};

constexpr int kInvBlocks = 1024;

// Device tables of the two-level preconditioner (see PrecondArgs), float64 and float32.
struct PcTables {
  double* Bt = nullptr;
  Cplx<double>*twx = nullptr, *twy = nullptr;
  double *ax = nullptr, *ay = nullptr;
  float* Btf = nullptr;
  Cplx<float>*twxf = nullptr, *twyf = nullptr;
  float *axf = nullptr, *ayf = nullptr;
  int log2x = -1, log2y = -1;
  // spectral preconditioner (periodic grids): eigenvectors and eigenvalues of the 1D symbols
  Cplx<double>*Vx = nullptr, *Vy = nullptr;
  double *lx = nullptr, *ly = nullptr;
  Cplx<float>*Vxf = nullptr, *Vyf = nullptr;
  float *lxf = nullptr, *lyf = nullptr;
  int spectral_rc = DG_ERR_ARG;  // DG_OK once the spectral tables are built
};

struct dg_grid {
  int Nx, Ny, n;
  double Lx, Ly, hx, hy, tau;
  int bc = 0;  // DG_BC_PERIODIC or DG_BC_DIRICHLET
  RefTables rt;
  int rTY, rTX, cTY, cTX;
  int num_sms;
  OpsHost ops;
  Workspace ws;
  int precond = 0;  // DG_PRECOND_JACOBI, DG_PRECOND_TWOLEVEL or DG_PRECOND_SPECTRAL
  bool cluster_ok = true;  // small solves may run as one thread-block cluster
  PcTables pc;
  void* d_opsd = nullptr;  // device copies of the operator tables (batched kernel)
  void* d_opsf = nullptr;
  void* d_opsx = nullptr;  // Ops2D<df, n>
  void* d_opsk = nullptr;  // OpsK<df, n>
  // a float32 evaluation of the CG operator is too inexact on the smoothest modes of this grid
  // (see precise_apply_needed): mixed solves apply it in double-float
  int precise_apply = 0;  // 0 float32, 1 double-float, 2 adaptive (MixedArgs::precise_apply)
  int precise_auto = 0;   // the automatic choice (dg_grid_set_compensated_apply(g, -1))
  // float64 rounding floor of the CG residual per unit y.y, (2^-52 x the row-sum bound of
  // |Ahat|)^2: solves accept a residual below max(tol^2 b.b, floor2 y.y)
  double floor2 = 0.0;
};

struct dg_sim {
  dg_grid* g;
  long long batch_limit = 0;  // batched steps stop at this step index (0: no limit)
  double D, dt, tol;
  int precision, maxit, fixed_iters;
  long long step;
  double* omega[2];
  int oc;
  double* psi[3];  // scaled: sqrt(W) psi
  int p0, p1, p2;
  // Ahat applied to each psi slot, valid where apsi_ok: every tolerance-stopped solve ends with
  // the true residual of its result, whose operator product is kept, so that the next solve's
  // initial residual b - Ahat (2 psi^k - psi^{k-1}) needs no operator application
  double* apsi[3] = {nullptr, nullptr, nullptr};
  bool apsi_ok[3] = {false, false, false};
  void* R[4];      // history ring: float64 (DG_FP64) or float32 (DG_MIXED)
  int r1, r2, r3, rfree;  // R^{k-1}, R^{k-2}, R^{k-3}, free slot
  int K = 3;              // steps of the Adams-Bashforth method (1..4)
  int parts = 0;          // bracket parts (0: J of Eq. J; 1: J++ alone, the naive bracket)
  double *stA, *stB;  // RK stage vorticities
  void *k2, *k3;      // RK stage slopes (same type as R)
  double tol_in;      // inner relative tolerance of the float32 sweeps (DG_MIXED)
  int max_sweeps;
  Workspace ws;
  // launch accounting / device timing
  long long launches = 0, rhs_launches = 0, cg_launches = 0;
  bool timing = false;
  std::vector<cudaEvent_t> ev_rhs, ev_cg;  // start/stop pairs
  size_t n_ev_rhs = 0, n_ev_cg = 0;
};

namespace dgk {

inline size_t ndof_of(const dg_grid* g) { return (size_t)g->Nx * g->Ny * g->n * g->n; }

inline Geom geom_of(const dg_grid* g, int TY, int TX) {
  Geom G;
  G.Nx = g->Nx;
  G.Ny = g->Ny;
  G.TY = std::min(TY, g->Ny);
  G.TX = std::min(TX, g->Nx);
  G.tilesX = (g->Nx + G.TX - 1) / G.TX;
  G.tilesY = (g->Ny + G.TY - 1) / G.TY;
  G.bc = g->bc;
  return G;
}

template <typename T, int N>
const Ops2D<T, N>& ops_of(const dg_grid* g) {
  if constexpr (std::is_same<T, double>::value) return *reinterpret_cast<const Ops2D<T, N>*>(g->ops.d);
  else if constexpr (std::is_same<T, float>::value) return *reinterpret_cast<const Ops2D<T, N>*>(g->ops.f);
  else return *reinterpret_cast<const Ops2D<T, N>*>(g->ops.x);
}

template <int N>
const OpsK<df, N>& opsk_of(const dg_grid* g) {
  return *reinterpret_cast<const OpsK<df, N>*>(g->ops.k);
}

template <class F>
int dispatch_n(int n, F&& f) {
  switch (n) {
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    case 3: return f(std::integral_constant<int, 3>{});
    case 4: return f(std::integral_constant<int, 4>{});
    case 5: return f(std::integral_constant<int, 5>{});
  }
  return fail(DG_ERR_ARG, "n = %d outside 1..5", n);
}

template <typename Kern>
int set_smem(Kern k, size_t bytes) {
  // above 48 KB of static plus dynamic shared memory a kernel must opt in; our kernels' static
  // shared memory is well under 16 KB
  if (bytes > 32 * 1024) CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  return DG_OK;
}

// Both cell counts are powers of two (the DFTs run in place, without a second line buffer).
inline bool pow2_grid(const dg_grid* g) { return g->pc.log2x >= 0 && g->pc.log2y >= 0; }

inline PrecondArgs<double> pc_args(const dg_grid* g, const Workspace& w) {
  PrecondArgs<double> P{};
  P.kind = g->precond;
  P.Vx = g->pc.Vx;
  P.lx = g->pc.lx;
  P.Vy = g->pc.Vy;
  P.ly = g->pc.ly;
  P.S = w.pS;
  P.Bt = g->pc.Bt;
  P.twx = g->pc.twx;
  P.twy = g->pc.twy;
  P.ax = g->pc.ax;
  P.ay = g->pc.ay;
  P.log2x = g->pc.log2x;
  P.log2y = g->pc.log2y;
  P.z = w.pz;
  P.rc = w.prc;
  P.uc = w.puc;
  P.C = w.pC;
  return P;
}

inline PrecondArgs<float> pc_args_f(const dg_grid* g, const Workspace& w) {
  PrecondArgs<float> P{};
  P.kind = g->precond;
  P.Vx = g->pc.Vxf;
  P.lx = g->pc.lxf;
  P.Vy = g->pc.Vyf;
  P.ly = g->pc.lyf;
  P.S = w.pSf;
  P.Bt = g->pc.Btf;
  P.twx = g->pc.twxf;
  P.twy = g->pc.twyf;
  P.ax = g->pc.axf;
  P.ay = g->pc.ayf;
  P.log2x = g->pc.log2x;
  P.log2y = g->pc.log2y;
  P.z = w.pzf;
  P.rc = w.prcf;
  P.uc = w.pucf;
  P.C = w.pCf;
  return P;
}

// Records the next event of a start/stop pool (growing it as needed).
inline int record_event(std::vector<cudaEvent_t>& pool, size_t& used, cudaStream_t st) {
  if (used == pool.size()) {
    cudaEvent_t e;
    CUDA_TRY(cudaEventCreate(&e));
    pool.push_back(e);
  }
  CUDA_TRY(cudaEventRecord(pool[used++], st));
  return DG_OK;
}

// Small grids: if the built-in tiles of n cover the grid with at most kClusterMax tiles, the
// mixed-precision solve (float32 inner iterations: latency-bound, not throughput-bound) runs
// as ONE thread-block cluster of that many blocks, whose phases meet at the hardware cluster
// barrier instead of the grid barrier in global memory.  The float64 solve, bound by the
// float64 FMA rate, keeps the whole GPU (small tiles, cooperative launch): on 32^2 cells, n = 3,
// a cluster of 8 blocks took 66 us per float64 iteration against 46 us on 256 tiles, while
// the mixed solve ran twice as fast as a cluster.
constexpr int kClusterMax = 8;  // the portable cluster size

inline Geom solve_geom(const dg_grid* g, bool allow_cluster, bool* cluster) {
  int rty, rtx, cty, ctx;
  default_tiles(g->n, rty, rtx, cty, ctx);
  const Geom Gd = geom_of(g, cty, ctx);
  *cluster = allow_cluster && g->cluster_ok && Gd.tilesX * Gd.tilesY <= kClusterMax;
  return *cluster ? Gd : geom_of(g, g->cTY, g->cTX);
}

inline int co_resident_cap(const dg_grid* g) { return std::max(64, 8 * g->num_sms); }

// ---- per-n kernel launchers (dg_launch.cuh; instantiated in dg_inst_n<N>.cu) -------------
template <typename T, int N>
int launch_rhs(const dg_grid* g, const RhsArgs<T>& A, cudaStream_t st);
template <typename T, int N>
int launch_apply(const dg_grid* g, const double* x, double* y, int mode, cudaStream_t st);
template <typename T, int N, typename TP = T>
int launch_cg(const dg_grid* g, CgArgs<T, TP> A, const Workspace& w, cudaStream_t st, dg_sim* timed = nullptr);
template <int N>
int launch_mixed(const dg_grid* g, MixedArgs A, const Workspace& w, cudaStream_t st, dg_sim* timed = nullptr);
template <int N>
int launch_invariants(const dg_grid* g, const double* psi, const double* omega, int psi_scaled, const Workspace& w,
                      cudaStream_t st);
// y[i] = x[i] * sqrt(W) (inverse = 0) or x[i] / sqrt(W) (inverse = 1), per node
template <int N>
int launch_scale(const dg_grid* g, const double* x, double* y, int inverse, cudaStream_t st);

// ---- launchers of the n-independent kernels (dg_misc.cu, dg_batch.cu) ------------------
int launch_invariants_final(const double* part, int nparts, double* out, cudaStream_t st);
// the capped-barrier self-test kernel; returns the CUDA error of the launch
cudaError_t launch_barrier_selftest(SyncState* s, int* out, cudaStream_t st);
// the batched persistent kernel: occupancy for smem bytes of dynamic shared memory, launch
int batch_kernel_occupancy(size_t smem, int* per_sm);
int batch_kernel_launch(const BatchArgs& A, int grid, size_t smem, cudaStream_t st);

}  // namespace dgk
