// The batched persistent kernel (many simulations per cooperative launch) and its launch.
#include "dg_host.cuh"

namespace dgk {

__global__ void __launch_bounds__(kThreads) batch_kernel(const __grid_constant__ BatchArgs A) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ double redd[32];
  __shared__ double bcd;
  __shared__ float redf[32];
  __shared__ float bcf;
  __shared__ int s_flag;
  int gi = 0;
  while (gi + 1 < A.ngroups && (int)blockIdx.x >= A.groups[gi + 1].first_block) ++gi;
  const BatchGroup grp = A.groups[gi];
  const int vrank = int(blockIdx.x) - grp.first_block;
  bool ok = true;
  for (int st = 0; st < A.nsteps && ok; ++st) {
    for (int j = 0; j < grp.count && ok; ++j) {
      BatchSim* S = A.sims + A.order[grp.first + j];
      switch (S->n) {
        case 1: ok = batch_step<1>(S, grp, vrank, smem_raw, redd, &bcd, redf, &bcf, &s_flag); break;
        case 2: ok = batch_step<2>(S, grp, vrank, smem_raw, redd, &bcd, redf, &bcf, &s_flag); break;
        case 3: ok = batch_step<3>(S, grp, vrank, smem_raw, redd, &bcd, redf, &bcf, &s_flag); break;
        case 4: ok = batch_step<4>(S, grp, vrank, smem_raw, redd, &bcd, redf, &bcf, &s_flag); break;
        case 5: ok = batch_step<5>(S, grp, vrank, smem_raw, redd, &bcd, redf, &bcf, &s_flag); break;
        default: ok = false;
      }
    }
  }
  if (!ok && threadIdx.x == 0) atomicCAS(A.error, 0, kFlagTimeout);
}

int batch_kernel_occupancy(size_t smem, int* per_sm) {
  if (int rc = set_smem(batch_kernel, smem)) return rc;
  CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, batch_kernel, kThreads, smem));
  return DG_OK;
}

int batch_kernel_launch(const BatchArgs& A, int grid, size_t smem, cudaStream_t st) {
  // cudaLaunchKernelEx with the cooperative attribute: the form of a cooperative launch
  // that stream capture (and so the CUDA graph) accepts.
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CUDA_TRY(cudaLaunchKernelEx(&cfg, batch_kernel, A));
  return DG_OK;
}

}  // namespace dgk
