// Internal interface of the sampled-trace-kernel convolution C.
#pragma once

#include "pair_ops.cuh"

namespace mpi {

// Scratch bytes for the sampled kernel of a grid (FP64 copy + rounded copy).
size_t conv_kernel_bytes(int nx, int ny, int elem_bytes);

// Samples kappa_G on all (2ny-1) x (2nx-1) voxel offsets into `scratch`
// (conv_kernel_bytes) and returns the kernel in type R through K_out.
// comp < 0: the trace kernel; comp = 2a + b: entry (a, b) of beta K G.
template <typename R>
int conv_prepare_kernel(const ModelH &m, const GridH &g, void *scratch, R **K_out, cudaStream_t st,
                        int comp = -1);

// out = C in  (in: IN [ny][nx], out: OUT [ny][nx], must not overlap).
template <typename R, typename IN, typename OUT>
int launch_conv(const GridH &g, const R *K, const IN *in, OUT *out, cudaStream_t st);

}  // namespace mpi
