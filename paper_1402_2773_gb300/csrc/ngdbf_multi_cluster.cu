// ngdbf_multi_cluster.cu -- the job-table NGDBF kernel with thread-block clusters: codes of
// many symbols are split over the CTAs of a cluster, which exchange decision words through
// distributed shared memory (see decode_job).
#include "ngdbf_kernels.cuh"
#include "ngdbf_multi.h"

namespace ngdbf {

// The job table with thread-block clusters: the CTAs of a cluster start on the same job and
// move between jobs together.  A job with n >= A.split_min_n is split over the cluster (each
// CTA decodes a range of the symbols of the same 32 slots, see decode_job), shortening the
// time per iteration of its frames; a smaller job is decoded by each CTA of the cluster on its
// own slots.  Rank 0 picks the next job for the cluster once every CTA has finished this one.
template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE, int PREC>
__global__ void __launch_bounds__(1024) ngdbf_multi_cluster_kernel(const __grid_constant__ MultiArgs A) {
    using HeldT = typename Held<PREC>::T;
    cooperative_groups::cluster_group cluster = cooperative_groups::this_cluster();
    __shared__ Job job;
    __shared__ int32_t next_job;
    const int C = (int)cluster.num_blocks(), rank = (int)cluster.block_rank();
    HeldT* ys = static_cast<HeldT*>(A.yslots) + (size_t)blockIdx.x * pad4(A.n_local) * kSlots;
    uint16_t* st = A.st_global ? A.st_global + (size_t)blockIdx.x * pad4(A.n_local) * kSlots : nullptr;
    int j = A.first_job[blockIdx.x / C];
    while (j >= 0) {
        if (threadIdx.x == 0) job = A.jobs[j];
        __syncthreads();
        const bool sp = job.n >= A.split_min_n;
        const Split S = sp ? split_range(rank, C, job.n) : Split{0, 1, 0, job.n};
        // shared memory laid out for this job's share of symbols (the same in every CTA of
        // the cluster, so peer addresses agree)
        int tables = 0;
        const SmemLayout L = job_layout(job.n, job.m, job.t_max, job.dv_max, job.dc_max, ADAPT,
                                        ST_SMEM && (ADAPT || SMOOTH), WIDE, A.placement,
                                        sp ? split_local_max(job.n, C) : job.n, A.smem_bytes, &tables);
        decode_job<ADAPT, SMOOTH, ST_SMEM, WIDE, PREC, true>(job, job.thr, A.G, L, tables, ys, st, S);
        cluster.sync();
        if (rank == 0 && threadIdx.x == 0) {
            long long best = 0;
            int pick = -1;
            for (int i = 0; i < A.n_jobs; ++i) {
                const unsigned long long claimed = *(volatile unsigned long long*)A.jobs[i].queue;
                const long long left = A.jobs[i].n_frames - (long long)min(claimed, (unsigned long long)A.jobs[i].n_frames);
                // its estimated remaining work: unclaimed frames x work per frame
                const long long work = left * A.jobs[i].work;
                if (work > best) {
                    best = work;
                    pick = i;
                }
            }
            for (int r = 0; r < C; ++r) *cluster.map_shared_rank(&next_job, r) = pick;
        }
        cluster.sync();
        j = next_job;
    }
}

namespace {

using MultiFn = void (*)(MultiArgs);

template <bool AD, bool SM, int PREC>
MultiFn pick_width_cl(bool st_smem, bool wide) {
    if (st_smem) return wide ? ngdbf_multi_cluster_kernel<AD, SM, true, true, PREC> : ngdbf_multi_cluster_kernel<AD, SM, true, false, PREC>;
    return wide ? ngdbf_multi_cluster_kernel<AD, SM, false, true, PREC> : ngdbf_multi_cluster_kernel<AD, SM, false, false, PREC>;
}

template <int PREC>
MultiFn pick_variant_cl(int variant, bool st_smem, bool wide) {
    switch (variant & 3) {
        case 0: return pick_width_cl<false, false, PREC>(st_smem, wide);
        case 1: return pick_width_cl<true, false, PREC>(st_smem, wide);
        case 2: return pick_width_cl<false, true, PREC>(st_smem, wide);
        default: return pick_width_cl<true, true, PREC>(st_smem, wide);
    }
}

}  // namespace

void* multi_cluster_kernel_fn(int variant, int precision, bool st_smem, bool wide) {
    switch (precision) {
        case NGDBF_FP16: return (void*)pick_variant_cl<kFP16>(variant, st_smem, wide);
        case NGDBF_FIX: return (void*)pick_variant_cl<kFIX>(variant, st_smem, wide);
        case NGDBF_FIXACC: return (void*)pick_variant_cl<kFIXACC>(variant, st_smem, wide);
        default: return (void*)pick_variant_cl<kFP32>(variant, st_smem, wide);
    }
}

int max_active_clusters(void* fn, int cluster, int block, int smem) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)cluster);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
}

}  // namespace ngdbf
