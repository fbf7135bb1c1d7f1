// Definitions of the per-n kernel launchers declared in dg_host.cuh.  Included only by the
// dg_inst_n<N>.cu translation units, each of which instantiates them for one n.
#pragma once

#include "dg_host.cuh"

namespace dgk {

template <typename T, int N>
int launch_rhs(const dg_grid* g, const RhsArgs<T>& A, cudaStream_t st) {
  const Geom G = geom_of(g, g->rTY, g->rTX);
  const size_t smem = table_bytes<Ops2D<T, N>>() + rhs_smem_values<T, N>(G.TY, G.TX) * sizeof(T);
  if (int rc = set_smem(rhs_kernel<T, N>, smem)) return rc;
  rhs_kernel<T, N><<<G.tilesX * G.tilesY, rhs_threads<N>(), smem, st>>>(ops_of<T, N>(g), G, A);
  CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

template <typename T, int N>
int launch_apply(const dg_grid* g, const double* x, double* y, int mode, cudaStream_t st) {
  const Geom G = geom_of(g, g->cTY, g->cTX);
  const size_t smem = table_bytes<Ops2D<T, N>>() + apply_smem_values<T, N>(G.TY, G.TX) * sizeof(T);
  if (int rc = set_smem(apply_kernel<T, N>, smem)) return rc;
  apply_kernel<T, N><<<G.tilesX * G.tilesY, kThreads, smem, st>>>(ops_of<T, N>(g), G, x, y, mode);
  CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

// Launches kern with args on grid blocks: as one cluster (cluster == true; cooperative
// launch otherwise).  Returns false in *launched when the cluster does not fit (the caller
// then falls back to a cooperative launch).
template <class Kern, class... Args>
int launch_solve(Kern kern, bool cluster, int grid, size_t smem, cudaStream_t st, bool* launched, Args... args) {
  *launched = false;
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (cluster) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = grid;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int nclusters = 0;
    if (cudaOccupancyMaxActiveClusters(&nclusters, kern, &cfg) != cudaSuccess || nclusters < 1) {
      cudaGetLastError();
      return DG_OK;
    }
  } else {
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, args...));
  *launched = true;
  return DG_OK;
}

template <typename T, int N, typename TP>
int launch_cg(const dg_grid* g, CgArgs<T, TP> A, const Workspace& w, cudaStream_t st, dg_sim* timed) {
  bool cluster = false;
  Geom G = solve_geom(g, false, &cluster);
  size_t smem = table_bytes<Ops2D<T, N>>() + cg_smem_bytes<T, N>(G.TY, G.TX, std::max(g->Nx, g->Ny), A.precond, pow2_grid(g));
  auto kern = cg_kernel<T, N, TP>;
  if (int rc = set_smem(kern, smem)) return rc;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (A.precond == kPrecondSpectral && per_sm <= 2) {
    // the spectral line buffers leave room for two blocks per SM: the variant whose register
    // budget assumes two (no spills in the spectral transforms)
    kern = cg_kernel<T, N, TP, 2>;
    if (int rc = set_smem(kern, smem)) return rc;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  }
  if (per_sm < 1) return fail(DG_ERR_CUDA, "CG kernel does not fit on an SM (smem %zu B)", smem);
  int grid = std::min(per_sm * g->num_sms, G.tilesX * G.tilesY);
  grid = std::min(grid, w.grid_cap);
  A.part = reinterpret_cast<T*>(w.part);
  A.sync = w.sync;
  A.status = w.status;
  if constexpr (std::is_same<TP, double>::value)
    A.pc = pc_args(g, w);
  else
    A.pc = pc_args_f(g, w);
  CUDA_TRY(cudaMemsetAsync(w.sync, 0, sizeof(SyncState), st));
  const bool tm = timed && timed->timing;
  if (tm)
    if (int rc = record_event(timed->ev_cg, timed->n_ev_cg, st)) return rc;
  bool launched = false;
  A.cluster = cluster ? 1 : 0;
  if (int rc = launch_solve(kern, cluster, grid, smem, st, &launched, ops_of<T, N>(g), G, A)) return rc;
  if (!launched) {  // no room for the cluster: the tiles of a cooperative launch instead
    G = geom_of(g, g->cTY, g->cTX);
    smem = table_bytes<Ops2D<T, N>>() + cg_smem_bytes<T, N>(G.TY, G.TX, std::max(g->Nx, g->Ny), A.precond, pow2_grid(g));
    if (int rc = set_smem(kern, smem)) return rc;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    grid = std::min({per_sm * g->num_sms, G.tilesX * G.tilesY, w.grid_cap});
    A.cluster = 0;
    if (int rc = launch_solve(kern, false, grid, smem, st, &launched, ops_of<T, N>(g), G, A)) return rc;
  }
  if (tm)
    if (int rc = record_event(timed->ev_cg, timed->n_ev_cg, st)) return rc;
  return DG_OK;
}

template <int N>
int launch_mixed(const dg_grid* g, MixedArgs A, const Workspace& w, cudaStream_t st, dg_sim* timed) {
  bool cluster = false;
  Geom G = solve_geom(g, true, &cluster);
  auto smem_of = [&](const Geom& Gx) {
    return mixed_ops_bytes<N>() + mixed_smem_bytes<N>(Gx.TY, Gx.TX, std::max(g->Nx, g->Ny), A.precond, pow2_grid(g));
  };
  size_t smem = smem_of(G);
  auto kern = mixed_cg_kernel<N>;
  if (int rc = set_smem(kern, smem)) return rc;
  int per_sm = 0;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  if (A.precond == kPrecondSpectral && per_sm <= 2) {  // as in launch_cg
    kern = mixed_cg_kernel<N, 2>;
    if (int rc = set_smem(kern, smem)) return rc;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
  }
  if (per_sm < 1) return fail(DG_ERR_CUDA, "mixed CG kernel does not fit on an SM (smem %zu B)", smem);
  int grid = std::min(per_sm * g->num_sms, G.tilesX * G.tilesY);
  grid = std::min(grid, w.grid_cap);
  A.rf = w.rf;
  A.v = CgVectors<float>{w.fe, w.fr, w.fp0, w.fp1, w.fq};
  A.pc = pc_args_f(g, w);
  A.partd = w.part;
  A.partf = w.partf;
  A.sync = w.sync;
  A.status = w.status;
  CUDA_TRY(cudaMemsetAsync(w.sync, 0, sizeof(SyncState), st));
  const bool tm = timed && timed->timing;
  if (tm)
    if (int rc = record_event(timed->ev_cg, timed->n_ev_cg, st)) return rc;
  bool launched = false;
  A.cluster = cluster ? 1 : 0;
  if (int rc = launch_solve(kern, cluster, grid, smem, st, &launched, ops_of<double, N>(g), ops_of<float, N>(g), opsk_of<N>(g), G, A))
    return rc;
  if (!launched) {  // no room for the cluster: the tiles of a cooperative launch instead
    G = geom_of(g, g->cTY, g->cTX);
    smem = smem_of(G);
    if (int rc = set_smem(kern, smem)) return rc;
    CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    grid = std::min({per_sm * g->num_sms, G.tilesX * G.tilesY, w.grid_cap});
    A.cluster = 0;
    if (int rc = launch_solve(kern, false, grid, smem, st, &launched, ops_of<double, N>(g), ops_of<float, N>(g), opsk_of<N>(g), G, A))
      return rc;
  }
  if (tm)
    if (int rc = record_event(timed->ev_cg, timed->n_ev_cg, st)) return rc;
  return DG_OK;
}

template <int N>
int launch_invariants(const dg_grid* g, const double* psi, const double* omega, int psi_scaled, const Workspace& w,
                      cudaStream_t st) {
  const NodeWeights<N> W = make_weights<N>(g->rt, g->hx, g->hy);
  const size_t nd = ndof_of(g);
  const int blocks = (int)std::min<size_t>(kInvBlocks, (nd + kThreads - 1) / kThreads);
  invariants_partial_kernel<N><<<blocks, kThreads, 0, st>>>(W, psi, omega, nd, psi_scaled, w.inv_part);
  CUDA_TRY(cudaGetLastError());
  return launch_invariants_final(w.inv_part, blocks, w.inv_out, st);
}

template <int N>
int launch_scale(const dg_grid* g, const double* x, double* y, int inverse, cudaStream_t st) {
  const NodeWeights<N> W = make_weights<N>(g->rt, g->hx, g->hy);
  const size_t nd = ndof_of(g);
  const int blocks = (int)std::min<size_t>(4096, (nd + kThreads - 1) / kThreads);
  scale_nodes_kernel<N><<<blocks, kThreads, 0, st>>>(W, x, y, nd, inverse);
  CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

}  // namespace dgk

// Explicit instantiation of every launcher for one n (in namespace dgk).
#define DGK_INSTANTIATE_LAUNCHERS(N)                                                                           \
  namespace dgk {                                                                                             \
  template int launch_rhs<double, N>(const dg_grid*, const RhsArgs<double>&, cudaStream_t);                   \
  template int launch_rhs<df, N>(const dg_grid*, const RhsArgs<df>&, cudaStream_t);                           \
  template int launch_apply<double, N>(const dg_grid*, const double*, double*, int, cudaStream_t);            \
  template int launch_cg<double, N, double>(const dg_grid*, CgArgs<double, double>, const Workspace&,         \
                                            cudaStream_t, dg_sim*);                                           \
  template int launch_cg<double, N, float>(const dg_grid*, CgArgs<double, float>, const Workspace&,           \
                                           cudaStream_t, dg_sim*);                                            \
  template int launch_mixed<N>(const dg_grid*, MixedArgs, const Workspace&, cudaStream_t, dg_sim*);           \
  template int launch_invariants<N>(const dg_grid*, const double*, const double*, int, const Workspace&,      \
                                    cudaStream_t);                                                            \
  template int launch_scale<N>(const dg_grid*, const double*, double*, int, cudaStream_t);                    \
  }
