// ngdbf_host.h -- host-side pieces shared by the translation units of the C ABI
// (single decodes and job tables in ngdbf_decode.cu, the serving loop in ngdbf_server.cu).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/ngdbf.h"
#include "ngdbf_kernels.cuh"
#include "ngdbf_multi.h"

// Device-resident tables of one parity-check matrix.
struct ngdbf_code {
    int32_t n, m, dv_max, dc_max;
    int device;
    uint16_t* d_chk_cols;   // [dc_max][m] N(i) column-major, padded with n
    uint16_t* d_sym_chks;   // [n][dv_max] M(k) row-major, padded with m
    uint8_t* d_sym_deg;     // [n]
};

namespace ngdbf {
namespace host {

// Error text for the calling thread; returns s.
ngdbf_status fail(ngdbf_status s, const std::string& msg);
ngdbf_status cuda_fail(cudaError_t e, const char* what);
// Launch shape reported by ngdbf_last_launch on the calling thread.
void set_last_launch(int grid, int block, int smem, int state_in_smem, int tables_in_smem, int kernels,
                     int sm_count);
size_t align256(size_t v);
// The library's stream-ordered pool of a device (kept warm across calls).
ngdbf_status get_pool(int dev, cudaMemPool_t* out);
// Philox round keys and series coefficients of the perturbation generator.
void host_gen_consts(uint64_t seed, GenConsts& G);
// Bytes of one held sample of a precision.
size_t held_bytes(int precision);
ngdbf_status check_params(const ngdbf_params* P, float sigma);
// Shared-memory plan of a kernel of the slot loop for the given maxima: per-slot state in
// shared memory when it fits (fn_st) else global (fn_nost), adjacency tables, block size.
struct SmemPlan {
    bool st_smem;
    int placement, block, bps, smem;
};
ngdbf_status plan_smem(int dev, int n, int m, int t_max, int dv_max, int dc_max, bool adapt, bool state,
                       const void* fn_st, const void* fn_nost, SmemPlan* out);
// Job fields and its threshold words thr[0..t_max].
void fill_job(const ngdbf_code* C, const ngdbf_params* P, const float* y, int64_t n_frames, float sigma,
              uint64_t frame_offset, uint8_t* bits, int32_t* iters, uint8_t* pass,
              unsigned long long* queue, Job* out, uint32_t* thr);

// Shared-memory plan of a job table: launch maxima, kernel, and candidate
// (block, CTAs per SM) shapes.
struct TablePlan {
    int n_max = 0, m_max = 0, t_max = 0, dv_max = 0, dc_max = 0;
    int variant = 0, precision = 0, sm_count = 0, smem = 0;
    bool st_smem = false, wide = false, state_global = false;
    int placement = 0;          // adjacency tables in shared memory: kTabChk | kTabSym
    size_t thr_words = 0;
    void* fn = nullptr;
    std::vector<std::pair<int, int>> shapes;
};
ngdbf_status plan_table(const ngdbf_job* jobs, int32_t n_jobs, int dev, TablePlan* out);

// One candidate launch shape of a job table: kernel, block size, cluster size (jobs of at
// least split_min_n symbols split over a cluster), shared-memory plan (state placement,
// adjacency tables in shared memory, symbols held per CTA) and the largest resident grid.
struct TableShape {
    void* fn = nullptr;
    int block = 0, cluster = 1, grid_max = 0, smem = 0, placement = 0, n_local = 0, split_min_n = 0;
    bool st_smem = false, state_global = false;
};
// The candidates of a planned table over block size x cluster size x table placement; the
// first is the default (no cluster, the plan's own placement, the largest block).
ngdbf_status table_shapes(const TablePlan& T, const ngdbf_job* jobs, int32_t n_jobs, int dev,
                          std::vector<TableShape>* out);
// Staged host-to-device copies (ngdbf_hostmem.cu): a pair of page-locked staging buffers of
// kStageBytes with the events that free them, taken from and returned to a library cache.
constexpr size_t kStageBytes = 128ull << 20;
struct Staging;
int host_copy_mode();
Staging* staging_acquire(int dev);      // nullptr when none can be allocated
void staging_release(Staging* s);
// bytes from host src to device dst on stream st: host threads fill a free staging buffer,
// the device copies out of it; returns when the last piece is queued.
cudaError_t staged_h2d(Staging* s, void* dst, const void* src, size_t bytes, cudaStream_t st);

// First job of every CTA, in proportion to the estimated work of each job.
std::vector<int32_t> assign_ctas(const std::vector<int64_t>& frames, const std::vector<int64_t>& weight, int grid);
std::vector<int32_t> assign_ctas_capped(const std::vector<int64_t>& frames, const std::vector<int64_t>& weight,
                                        const std::vector<int64_t>& cap, int grid);

}  // namespace host
}  // namespace ngdbf
