// ngdbf_multi.cu -- the job-table NGDBF kernel: one persistent launch over several
// decode jobs (codes of different length, rate, degree and iteration limit).
#include "ngdbf_kernels.cuh"
#include "ngdbf_multi.h"

namespace ngdbf {

template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE, int PREC>
__global__ void __launch_bounds__(1024) ngdbf_multi_kernel(const __grid_constant__ MultiArgs A) {
    using HeldT = typename Held<PREC>::T;
    __shared__ Job job;
    __shared__ int32_t next_job;
    HeldT* ys = static_cast<HeldT*>(A.yslots) + (size_t)blockIdx.x * pad4(A.n_max) * kSlots;
    uint16_t* st = A.st_global ? A.st_global + (size_t)blockIdx.x * pad4(A.n_max) * kSlots : nullptr;
    int j = A.first_job[blockIdx.x];
    while (j >= 0) {
        if (threadIdx.x == 0) job = A.jobs[j];
        __syncthreads();
        // shared memory laid out for this job's code (the launch has room for the largest)
        int tables = 0;
        const SmemLayout L = job_layout(job.n, job.m, job.t_max, job.dv_max, job.dc_max, ADAPT,
                                        ST_SMEM && (ADAPT || SMOOTH), WIDE, A.placement, job.n, A.smem_bytes,
                                        &tables);
        decode_job<ADAPT, SMOOTH, ST_SMEM, WIDE, PREC>(job, job.thr, A.G, L, tables, ys, st);
        // the next job: the one with the most unclaimed work (none left: done)
        if (threadIdx.x == 0) {
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
            next_job = pick;
        }
        __syncthreads();
        j = next_job;
        __syncthreads();
    }
}


namespace {

using MultiFn = void (*)(MultiArgs);

template <bool AD, bool SM, int PREC>
MultiFn pick_width(bool st_smem, bool wide) {
    if (st_smem) return wide ? ngdbf_multi_kernel<AD, SM, true, true, PREC> : ngdbf_multi_kernel<AD, SM, true, false, PREC>;
    return wide ? ngdbf_multi_kernel<AD, SM, false, true, PREC> : ngdbf_multi_kernel<AD, SM, false, false, PREC>;
}

template <int PREC>
MultiFn pick_variant(int variant, bool st_smem, bool wide) {
    switch (variant & 3) {
        case 0: return pick_width<false, false, PREC>(st_smem, wide);
        case 1: return pick_width<true, false, PREC>(st_smem, wide);
        case 2: return pick_width<false, true, PREC>(st_smem, wide);
        default: return pick_width<true, true, PREC>(st_smem, wide);
    }
}

}  // namespace

void* multi_kernel_fn(int variant, int precision, bool st_smem, bool wide) {
    switch (precision) {
        case NGDBF_FP16: return (void*)pick_variant<kFP16>(variant, st_smem, wide);
        case NGDBF_FIX: return (void*)pick_variant<kFIX>(variant, st_smem, wide);
        case NGDBF_FIXACC: return (void*)pick_variant<kFIXACC>(variant, st_smem, wide);
        default: return (void*)pick_variant<kFP32>(variant, st_smem, wide);
    }
}

cudaError_t launch_multi(void* fn, const MultiArgs& args, int grid, int block, int smem, cudaStream_t stream) {
    if (args.cluster <= 1) {
        reinterpret_cast<MultiFn>(fn)<<<grid, block, smem, stream>>>(args);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)args.cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = (size_t)smem;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, reinterpret_cast<MultiFn>(fn), args);
}

}  // namespace ngdbf
