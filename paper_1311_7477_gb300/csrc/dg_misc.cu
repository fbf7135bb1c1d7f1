// The small n-independent kernels and their launches: the final stage of the invariant
// sums and the barrier self-test.
#include "dg_host.cuh"

namespace dgk {

// =========================================================================================
// Invariants, second stage: one warp adds the per-block partials in a fixed order.
// =========================================================================================
__global__ void invariants_final_kernel(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  __shared__ double bc;
  for (int j = 0; j < 3; ++j) {
    const double s = sum_partials(part + j, nparts, 3, &bc);
    if (threadIdx.x == 0) out[j] = (j == 0) ? s : 0.5 * s;
  }
}

// Self-test of the capped grid barrier: block 0 never arrives, so every other block's wait
// runs out after kSpinCap polls and raises kFlagTimeout; nothing faults or hangs.
__global__ void barrier_selftest_kernel(SyncState* s, int* out) {
  __shared__ int f;
  if (blockIdx.x == 0) return;
  const bool ok = grid_barrier(s, &f, gridDim.x);
  if (threadIdx.x == 0 && !ok) atomicOr(out, kFlagTimeout);
}

int launch_invariants_final(const double* part, int nparts, double* out, cudaStream_t st) {
  invariants_final_kernel<<<1, 32, 0, st>>>(part, nparts, out);
  CUDA_TRY(cudaGetLastError());
  return DG_OK;
}

cudaError_t launch_barrier_selftest(SyncState* s, int* out, cudaStream_t st) {
  void* args[] = {(void*)&s, (void*)&out};
  return cudaLaunchCooperativeKernel((const void*)barrier_selftest_kernel, dim3(4), dim3(64), args, 0, st);
}

}  // namespace dgk
