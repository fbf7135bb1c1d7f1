// The kernels and launchers of the hot path for n = 3 nodes per cell and dimension.
#include "dg_launch.cuh"

DGK_INSTANTIATE_LAUNCHERS(3)
