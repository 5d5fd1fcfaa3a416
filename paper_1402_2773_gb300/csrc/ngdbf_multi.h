// ngdbf_multi.h -- host-side entry to the job-table kernel (defined in ngdbf_multi.cu).
#pragma once

#include <cuda_runtime.h>

#include "ngdbf_kernels.cuh"

namespace ngdbf {

// The job-table kernel for a variant (NGDBF_ADAPT | NGDBF_SMOOTH | NGDBF_SINGLE), a precision,
// the placement of the per-slot state and the count layout (4-bit lanes for symbol degrees up to
// 7, bit slices above); usable with cudaFuncSetAttribute and the occupancy calculator.
void* multi_kernel_fn(int variant, int precision, bool st_smem, bool wide);

// The same with thread-block clusters (jobs with n >= MultiArgs::split_min_n split over a cluster).
void* multi_cluster_kernel_fn(int variant, int precision, bool st_smem, bool wide);

// Launches the job-table kernel `fn` on `stream` (a cluster launch when args.cluster > 1).
cudaError_t launch_multi(void* fn, const MultiArgs& args, int grid, int block, int smem, cudaStream_t stream);

// Clusters of `cluster` CTAs of `fn` that can be resident at once (0 if none).
int max_active_clusters(void* fn, int cluster, int block, int smem);

}  // namespace ngdbf
