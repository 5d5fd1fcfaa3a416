// ngdbf_decode.cu -- the single-job NGDBF kernel and the C ABI (validation, code tables,
// launch planning, host pipeline, job tables).  Device code shared with the job-table
// kernel lives in ngdbf_kernels.cuh.
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ngdbf.h"
#include "ngdbf_host.h"
#include "ngdbf_kernels.cuh"

namespace ngdbf {

// Deviates of consecutive Philox outputs r = start + i (verification entry point).
__global__ void gaussian_range_kernel(const __grid_constant__ GenConsts G, uint32_t start, uint32_t count,
                                      float* z) {
    __shared__ float4 tab[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = G.icdf[i];
    __syncthreads();
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
        z[i] = gauss_icdf(start + i, tab);
}

// Same-mix throughput probe: the per-slot work of the decode's symbol loop for `groups` groups of
// four symbols on register-resident data (one Philox call, four inverse-CDF deviates from the
// shared coefficient table, the FP32 inversion function from a 4-bit count lane, the threshold
// lookup in shared memory and the comparison, the adaptation and window counters, and a warp
// ballot rebuilding the decision word), without the sample, state and count traffic.  Every
// thread folds its result into *sink so that nothing is dead code.
__global__ void __launch_bounds__(256) mix_probe_kernel(const __grid_constant__ GenConsts G, int groups, uint32_t* sink) {
    __shared__ float4 tab[256];
    __shared__ uint32_t thr[kMaxT + 1];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = G.icdf[i];
    for (int u = threadIdx.x; u <= kMaxT; u += blockDim.x) thr[u] = __float_as_uint(-0.7f + 0.001f * (float)u);
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t fid = blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t nib_shift = 4u * (lane & 7u);
    const float wgt = 0.1875f, wgt_m8 = -8.0f * 0.1875f, scale = 0.35f;
    uint32_t xw[4] = {0x0F0F0F0Fu ^ fid, 0x33333333u, 0x55555555u ^ fid, 0x00FF00FFu};
    uint32_t sv[4] = {lane, lane + 3u, lane + 7u, lane + 11u};
    uint32_t cw = 0x9ABCDEF1u ^ (fid << 4);
    const float yv[4] = {0.9f + 0.01f * lane, -0.2f, 1.3f, 0.45f};
    for (int g = 0; g < groups; ++g) {
        float z[4];
        noise4((uint32_t)g, 0u, fid, 0u, G, tab, false, z);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t th = thr[sv[j] & kUMask];
            const uint32_t nib = (cw >> nib_shift) & 0xFu;
            const float ws = __fmaf_rn(wgt, __uint2float_rn(nib), wgt_m8);
            const uint32_t xsign = (xw[j] << (31u - lane)) & 0x80000000u;
            const float q = __fmul_rn(scale, z[j]);
            const float E = __fadd_rn(__fadd_rn(__uint_as_float(__float_as_uint(yv[j]) ^ xsign), ws), q);
            const bool flip = E < __uint_as_float(th);
            sv[j] = (sv[j] + (flip ? 0u : 1u) + (xsign >> (31 - kCShift))) & 0x3FFFu;
            xw[j] ^= __ballot_sync(0xFFFFFFFFu, flip);
        }
        cw = (cw >> 4) | (cw << 28);
    }
    atomicXor(sink, xw[0] ^ xw[1] ^ xw[2] ^ xw[3] ^ sv[0] ^ sv[1] ^ sv[2] ^ sv[3]);
}

template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE, int PREC>
__global__ void __launch_bounds__(1024) ngdbf_persistent_kernel(const __grid_constant__ DecodeArgs A) {
    using HeldT = typename Held<PREC>::T;
    const Job& J = A.J;
    const SmemLayout L = smem_layout(J.n, J.m, J.t_max, J.dv_max, J.dc_max, ADAPT,
                                     ST_SMEM && (ADAPT || SMOOTH), A.placement);
    HeldT* ys = static_cast<HeldT*>(A.yslots) + (size_t)blockIdx.x * pad4(J.n) * kSlots;
    uint16_t* st = A.st_global ? A.st_global + (size_t)blockIdx.x * pad4(J.n) * kSlots : nullptr;
    decode_job<ADAPT, SMOOTH, ST_SMEM, WIDE, PREC>(J, A.thr, A.G, L, A.placement, ys, st);
}

}  // namespace ngdbf


// ===========================================================================
// Host side: validation, code tables, launch configuration, C ABI
// ===========================================================================

using namespace ngdbf;


namespace ngdbf {
namespace host {

thread_local std::string g_last_error;
thread_local ngdbf_launch_info g_last_launch = {0, 0, 0, 0, 0, 0};
thread_local ngdbf_host_stats g_last_host = {};

ngdbf_status fail(ngdbf_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

void set_last_launch(int grid, int block, int smem, int state_in_smem, int tables_in_smem, int kernels,
                     int sm_count) {
    g_last_launch.cluster = 1;
    g_last_launch.split_min_n = 0;
    g_last_launch.grid = grid;
    g_last_launch.block = block;
    g_last_launch.smem_bytes = smem;
    g_last_launch.state_in_smem = state_in_smem;
    g_last_launch.kernels = kernels;
    g_last_launch.sm_count = sm_count;
    g_last_launch.tables_in_smem = tables_in_smem;
}

size_t align256(size_t v) { return (v + 255) / 256 * 256; }

ngdbf_status cuda_fail(cudaError_t e, const char* what) {
    return fail(NGDBF_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// One stream-ordered pool per device for decode scratch; kept warm across calls.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

ngdbf_status get_pool(int dev, cudaMemPool_t* out) {
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (dev < 0 || dev >= 64) return fail(NGDBF_ERR_UNSUPPORTED, "device index out of range");
    if (!g_pools[dev]) {
        cudaMemPoolProps props;
        std::memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p;
        cudaError_t e = cudaMemPoolCreate(&p, &props);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemPoolCreate");
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = p;
    }
    *out = g_pools[dev];
    return NGDBF_OK;
}

namespace {

// Generator table of the inverse normal CDF (host, double precision, built once per process).
//
// Segment (j, s), j = 0..31, s = 0..7, covers the lower-tail probabilities
// p(v) = (8 + s + 1/2 + v) 2^-(j+5), v in [-1/2, 1/2].  Its FP32 cubic c0 + c1 v + c2 v^2 + c3 v^3
// is the polynomial through Phi^{-1} at the four Chebyshev points of [-1/2, 1/2],
// v_i = cos((2i+1) pi / 8) / 2, i = 0..3.  The definition fixes every double operation, so
// that an independent evaluation reproduces the FP32 words bit for bit:
//   * Phi^{-1}(p): 100 halvings of [-40, 0] on Phi(z) = erfc(-z / sqrt 2) / 2 (C library erfc),
//     keeping the half whose Phi at the midpoint is not below p as the upper end;
//   * with u = (cos(pi/8), cos(3 pi/8)) formed as sqrt(2 +- sqrt 2) / 2 and h = sqrt(2) / 2, the
//     nodes are (u0, u1, -u1, -u0) / 2; writing the node values as even parts e0 = g0 + g3,
//     e1 = g1 + g2 and odd parts o0 = g0 - g3, o1 = g1 - g2, the Chebyshev coefficients on
//     x = 2v are b0 = (e0 + e1) / 4, b1 = (o0 u0 + o1 u1) / 2, b2 = ((e0 - e1) h) / 2,
//     b3 = (o0 u1 - o1 u0) / 2, each in this order;
//   * T1(2v) = 2v, T2(2v) = 8v^2 - 1, T3(2v) = 32v^3 - 6v give the monomial coefficients
//     (b0 - b2, 2 b1 - 6 b3, 8 b2, 32 b3), rounded to FP32.
class InverseCdfTable {
  public:
    InverseCdfTable() {
        const double root2 = std::sqrt(2.0);
        u_[0] = 0.5 * std::sqrt(2.0 + root2);
        u_[1] = 0.5 * std::sqrt(2.0 - root2);
        h_ = 0.5 * root2;
        const double node[4] = {0.5 * u_[0], 0.5 * u_[1], -0.5 * u_[1], -0.5 * u_[0]};
        for (int seg = 0; seg < 256; ++seg) {
            const int level = seg >> 3, sub = seg & 7;
            double value[4];
            for (int i = 0; i < 4; ++i) value[i] = quantile(std::ldexp(8.0 + sub + 0.5 + node[i], -(level + 5)));
            words_[seg] = cubic(value);
        }
    }
    const float4* words() const { return words_; }

  private:
    static double lower_tail(double z) { return 0.5 * std::erfc(-z * 0.70710678118654752); }

    // Phi^{-1}(p) for 0 < p < 1/2 by interval halving on [-40, 0].
    static double quantile(double p) {
        double below = -40.0, above = 0.0;
        for (int step = 0; step < 100; ++step) {
            const double mid = 0.5 * (below + above);
            (lower_tail(mid) < p ? below : above) = mid;
        }
        return 0.5 * (below + above);
    }

    // Monomial coefficients of the cubic through the node values g (nodes in the order above).
    float4 cubic(const double g[4]) const {
        const double o0 = g[0] - g[3], o1 = g[1] - g[2];
        const double e0 = g[0] + g[3], e1 = g[1] + g[2];
        const double b0 = (e0 + e1) * 0.25;
        const double b1 = (o0 * u_[0] + o1 * u_[1]) * 0.5;
        const double b2 = ((e0 - e1) * h_) * 0.5;
        const double b3 = (o0 * u_[1] - o1 * u_[0]) * 0.5;
        return make_float4((float)(b0 - b2), (float)(2.0 * b1 - 6.0 * b3), (float)(8.0 * b2), (float)(32.0 * b3));
    }

    double u_[2], h_;
    float4 words_[256];
};

}  // namespace

const InverseCdfTable& icdf_table() {
    static const InverseCdfTable table;     // built once per process (thread-safe static)
    return table;
}

void host_gen_consts(uint64_t seed, GenConsts& G) {
    const InverseCdfTable& table = icdf_table();
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        G.rk0[r] = k0;
        G.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    std::memcpy(G.icdf, table.words(), sizeof(G.icdf));
}

struct LaunchPlan {
    int block, grid, blocks_per_sm, smem;
    bool st_smem;
    int placement;              // adjacency tables in shared memory: kTabChk | kTabSym
};

using KernelFn = void (*)(DecodeArgs);

template <bool AD, bool SM, int PREC>
KernelFn pick_width(bool st_smem, bool wide) {
    if (st_smem) return wide ? ngdbf_persistent_kernel<AD, SM, true, true, PREC> : ngdbf_persistent_kernel<AD, SM, true, false, PREC>;
    return wide ? ngdbf_persistent_kernel<AD, SM, false, true, PREC> : ngdbf_persistent_kernel<AD, SM, false, false, PREC>;
}

template <int PREC>
KernelFn pick_variant(int variant, bool st_smem, bool wide) {
    switch (variant & 3) {
        case 0: return pick_width<false, false, PREC>(st_smem, wide);
        case 1: return pick_width<true, false, PREC>(st_smem, wide);
        case 2: return pick_width<false, true, PREC>(st_smem, wide);
        default: return pick_width<true, true, PREC>(st_smem, wide);
    }
}

KernelFn pick_kernel(int variant, int precision, bool st_smem, bool wide) {
    switch (precision) {
        case NGDBF_FP16: return pick_variant<kFP16>(variant, st_smem, wide);
        case NGDBF_FIX: return pick_variant<kFIX>(variant, st_smem, wide);
        case NGDBF_FIXACC: return pick_variant<kFIXACC>(variant, st_smem, wide);
        default: return pick_variant<kFP32>(variant, st_smem, wide);
    }
}

// Bytes of one held sample.
size_t held_bytes(int precision) {
    return precision == NGDBF_FP16 ? 2 : ((precision == NGDBF_FIX || precision == NGDBF_FIXACC) ? 1 : 4);
}

// Shared-memory placement of a launch: the per-slot state and the adjacency tables.  The
// state stays in shared memory whenever some candidate fits with it there (it is read and
// written for every symbol and slot); among those candidates the most resident warps per
// SM win, then the most CTAs per SM, then more tables in shared memory (both, then the
// N(i) table alone).  fn_of(st) gives the kernel for a state placement.  Results are cached
// per shape and device.
struct PlacementChoice {
    bool st_smem = false;
    int placement = 0, block = 0, bps = 0;
    SmemLayout L{};
};

template <class FnOf>
ngdbf_status choose_placement(int dev, int n, int m, int t_max, int dv_max, int dc_max, bool adapt, bool state,
                              int limit, FnOf fn_of, PlacementChoice* out, int n_local = -1) {
    using Key = std::vector<int64_t>;
    static std::mutex mu;
    static std::map<Key, PlacementChoice> cache;
    const Key key = {dev, n, m, t_max, dv_max, dc_max, adapt, state, limit, n_local,
                     (int64_t)(intptr_t)fn_of(true), (int64_t)(intptr_t)fn_of(false)};
    {
        std::lock_guard<std::mutex> g(mu);
        auto it = cache.find(key);
        if (it != cache.end()) {
            *out = it->second;
            return NGDBF_OK;
        }
    }
    PlacementChoice best;
    int best_warps = 0;
    for (const bool st : {true, false}) {
        if (st && !state) continue;
        const void* fn = fn_of(st);
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        if (best.bps > 0) break;                       // state fits in shared memory
        for (const int tb : {kTabChk | kTabSym, kTabChk, 0}) {
            const SmemLayout L = smem_layout(n, m, t_max, dv_max, dc_max, adapt, st, tb, n_local);
            if (L.total > limit) continue;
            for (const int block : {1024, 512, 256}) {
                int bps = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, L.total);
                if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
                const int warps = bps * block / 32;
                if (bps > 0 && (warps > best_warps || (warps == best_warps && bps > best.bps))) {
                    best_warps = warps;
                    best.st_smem = st;
                    best.placement = tb;
                    best.block = block;
                    best.bps = bps;
                    best.L = L;
                }
            }
        }
    }
    if (best.bps == 0) return fail(NGDBF_ERR_UNSUPPORTED, "code too large for the shared-memory decision words");
    std::lock_guard<std::mutex> g(mu);
    cache[key] = best;
    *out = best;
    return NGDBF_OK;
}

ngdbf_status plan_smem(int dev, int n, int m, int t_max, int dv_max, int dc_max, bool adapt, bool state,
                       const void* fn_st, const void* fn_nost, SmemPlan* out) {
    int smem_optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, fn_nost);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    PlacementChoice pc;
    ngdbf_status s = choose_placement(dev, n, m, t_max, dv_max, dc_max, adapt, state,
                                      smem_optin - (int)fa.sharedSizeBytes,
                                      [&](bool st) { return st ? fn_st : fn_nost; }, &pc);
    if (s != NGDBF_OK) return s;
    out->st_smem = pc.st_smem;
    out->placement = pc.placement;
    out->block = pc.block;
    out->bps = pc.bps;
    out->smem = pc.L.total;
    return NGDBF_OK;
}

ngdbf_status plan_launch(const ngdbf_code* C, const ngdbf_params* P, int64_t n_frames, int dev,
                         LaunchPlan* plan, KernelFn* fn_out, int* sm_count_out) {
    int sm_count = 0, smem_optin = 0, smem_per_sm = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const bool state = (P->variant & 3) != 0;
    const bool adapt = (P->variant & NGDBF_ADAPT) != 0;
    const bool wide = C->dv_max > 7;
    PlacementChoice pc;
    ngdbf_status s = choose_placement(dev, C->n, C->m, P->t_max, C->dv_max, C->dc_max, adapt, state, smem_optin,
                                      [&](bool st) { return (const void*)pick_kernel(P->variant, P->precision, st, wide); },
                                      &pc);
    if (s != NGDBF_OK) return s;
    KernelFn fn = pick_kernel(P->variant, P->precision, pc.st_smem, wide);
    const int best_block = pc.block, best_bps = pc.bps;
    const SmemLayout& L = pc.L;
    const bool st_smem = pc.st_smem;
    const int placement = pc.placement;
    const int64_t groups = (n_frames + kSlots - 1) / kSlots;
    plan->block = best_block;
    plan->blocks_per_sm = best_bps;
    plan->grid = (int)std::min<int64_t>((int64_t)sm_count * best_bps, groups);
    plan->smem = L.total;
    plan->st_smem = st_smem;
    plan->placement = placement;
    *fn_out = fn;
    *sm_count_out = sm_count;
    (void)smem_per_sm;
    return NGDBF_OK;
}

// Standard deviation of the perturbation: fl32(eta sigma), or fl32(eta sigma sqrt 3) for the
// uniform deviates on (-1, 1) (same variance), formed in double.
float noise_scale(const ngdbf_params* P, float sigma) {
    const double s = (double)P->eta * (double)sigma;
    return (float)((P->variant & NGDBF_UNIFORM) ? s * std::sqrt(3.0) : s);
}

// FIXACC: accumulator steps per unit, fl32(2^(Q+8) / Y_max), and v in steps, rint(fl32(v Rd)).
float acc_scale(const ngdbf_params* P) { return (float)(std::ldexp(1.0, P->q_bits + kAccBits) / (double)P->y_max); }
int32_t acc_steps(float v, float Rd) {
    const float a = v * Rd;
    return (int32_t)std::lrint(a);
}

// Job fields of one decode and its threshold words thr[0..t_max].
void fill_job(const ngdbf_code* C, const ngdbf_params* P, const float* y, int64_t n_frames, float sigma,
              uint64_t frame_offset, uint8_t* bits, int32_t* iters, uint8_t* pass,
              unsigned long long* queue, Job* out, uint32_t* thr) {
    Job& J = *out;
    std::memset(&J, 0, sizeof(J));
    J.n = C->n; J.m = C->m; J.dv_max = C->dv_max; J.dc_max = C->dc_max;
    J.chk_cols = C->d_chk_cols; J.sym_chks = C->d_sym_chks; J.sym_deg = C->d_sym_deg;
    J.y = y; J.n_frames = n_frames; J.frame_offset = frame_offset;
    J.bits = bits; J.iters = iters; J.pass = pass; J.nb = (C->n + 7) / 8;
    J.w = P->precision == NGDBF_FP16 ? __half2float(__float2half_rn(P->w)) : P->w;
    J.scale = noise_scale(P, sigma);
    J.uniform = (P->variant & NGDBF_UNIFORM) ? 1 : 0;
    J.clamp = (P->y_max > 0.0f && std::isfinite(P->y_max)) ? 1 : 0;
    J.y_max = J.clamp ? P->y_max : 0.0f;
    J.t_max = P->t_max;
    J.t_smooth = std::max(0, P->t_max - P->smooth_window);
    J.queue = queue;
    J.work = (long long)C->n * (P->t_max + 1);
    J.single = (P->variant & NGDBF_SINGLE) ? 1 : 0;
    if (P->precision == NGDBF_FIX || P->precision == NGDBF_FIXACC) {
        J.fix_R = (float)(std::ldexp(1.0, P->q_bits) / (2.0 * (double)P->y_max));
        J.fix_kmax = (1 << (P->q_bits - 1)) - 1;
        J.fix_W = 2 * fix_code(P->w, J.fix_R, J.fix_kmax) + 1;
        J.trace_yunit = std::ldexp((double)P->y_max, -P->q_bits);
    }
    if (P->precision == NGDBF_FIXACC) {
        J.acc_R = acc_scale(P);
        J.acc_W = acc_steps(P->w, J.acc_R);
    }
    double p = 1.0;
    for (int u = 0; u <= P->t_max; ++u) {
        const float th = (float)((double)P->theta * p);      // fl32(theta lambda^u)
        uint32_t word;
        if (P->precision == NGDBF_FIX) {
            const int32_t v = 2 * fix_code(th, J.fix_R, J.fix_kmax) + 1;
            std::memcpy(&word, &v, 4);
        } else if (P->precision == NGDBF_FIXACC) {
            const int32_t v = acc_steps(th, J.acc_R);
            std::memcpy(&word, &v, 4);
        } else {
            const float h = P->precision == NGDBF_FP16 ? __half2float(__float2half_rn(th)) : th;
            std::memcpy(&word, &h, 4);
        }
        thr[u] = word;
        p = p * (double)P->lambda;
    }
}

// Kernel arguments of one decode: scratch at `base` (work counter, then the
// per-slot samples), per-slot state at `st_base` when it lives in global memory.
void fill_args(const ngdbf_code* C, const ngdbf_params* P, const LaunchPlan& plan, const float* y,
               int64_t n_frames, float sigma, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
               int32_t* iters, uint8_t* pass, unsigned char* base, unsigned char* st_base,
               bool st_global, DecodeArgs* out) {
    DecodeArgs& A = *out;
    std::memset(&A, 0, sizeof(A));
    fill_job(C, P, y, n_frames, sigma, frame_offset, bits, iters, pass,
             reinterpret_cast<unsigned long long*>(base), &A.J, A.thr);
    A.J.thr = nullptr;                 // thresholds travel inline in the launch
    A.placement = plan.placement;
    A.yslots = base + 256;
    A.st_global = st_global ? reinterpret_cast<uint16_t*>(st_base) : nullptr;
    host_gen_consts(seed, A.G);
}

ngdbf_status check_params(const ngdbf_params* P, float sigma) {
    if (!P) return fail(NGDBF_ERR_INVALID_ARG, "params is NULL");
    if (!(P->w > 0.0f) || !std::isfinite(P->w)) return fail(NGDBF_ERR_INVALID_ARG, "w must be finite and > 0");
    if (!std::isfinite(P->theta)) return fail(NGDBF_ERR_INVALID_ARG, "theta must be finite");
    if (!(P->eta >= 0.0f && P->eta <= 1.0f)) return fail(NGDBF_ERR_INVALID_ARG, "eta must be in [0, 1]");
    if (!(P->lambda > 0.0f && P->lambda <= 1.0f)) return fail(NGDBF_ERR_INVALID_ARG, "lambda must be in (0, 1]");
    if (std::isnan(P->y_max)) return fail(NGDBF_ERR_INVALID_ARG, "y_max is NaN");
    if (!(sigma >= 0.0f) || !std::isfinite(sigma)) return fail(NGDBF_ERR_INVALID_ARG, "sigma must be finite and >= 0");
    if (P->t_max < 0) return fail(NGDBF_ERR_INVALID_ARG, "t_max must be >= 0");
    if (P->t_max > NGDBF_MAX_T) return fail(NGDBF_ERR_UNSUPPORTED, "t_max above NGDBF_MAX_T");
    if (P->smooth_window < 0) return fail(NGDBF_ERR_INVALID_ARG, "smooth_window must be >= 0");
    if (P->smooth_window > NGDBF_MAX_WINDOW) return fail(NGDBF_ERR_UNSUPPORTED, "smooth_window above NGDBF_MAX_WINDOW");
    if (P->variant & ~15) return fail(NGDBF_ERR_INVALID_ARG, "unknown variant bits");
    if ((P->variant & NGDBF_SINGLE) && (P->variant & NGDBF_ADAPT))
        return fail(NGDBF_ERR_INVALID_ARG, "the single-bit variant has no threshold to adapt");
    if (P->precision < NGDBF_FP32 || P->precision > NGDBF_FIXACC) return fail(NGDBF_ERR_INVALID_ARG, "unknown precision");
    if (P->precision == NGDBF_FIX || P->precision == NGDBF_FIXACC) {
        if (P->q_bits < 2 || P->q_bits > 8) return fail(NGDBF_ERR_INVALID_ARG, "fixed point needs 2 <= q_bits <= 8");
        if (!(P->y_max > 0.0f) || !std::isfinite(P->y_max))
            return fail(NGDBF_ERR_INVALID_ARG, "fixed point needs a finite y_max > 0 (it sets the step)");
    } else if (P->q_bits != 0) {
        return fail(NGDBF_ERR_INVALID_ARG, "q_bits must be 0 unless precision is NGDBF_FIX or NGDBF_FIXACC");
    }
    if (P->precision == NGDBF_FIXACC) {
        // every accumulator term far inside int32: |theta|, 64 w and the largest perturbation
        // (8 standard deviations) below 2^28 steps
        const double Rd = acc_scale(P), lim = std::ldexp(1.0, 28);
        if (!(std::fabs((double)P->theta) * Rd < lim && (double)P->w * Rd * 64.0 < lim &&
              8.0 * (double)noise_scale(P, sigma) * Rd < lim))
            return fail(NGDBF_ERR_UNSUPPORTED, "NGDBF_FIXACC: theta, w or the perturbation exceeds the accumulator range");
    }
    return NGDBF_OK;
}

// Objective-trace buffers of one decode (ngdbf_decode_trace).
struct TraceSpec {
    int64_t frames;
    int32_t* unsat;
    int64_t* corr;
};

ngdbf_status decode_impl(const ngdbf_code* C, const float* y, int64_t n_frames, float sigma,
                         const ngdbf_params* P, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
                         int32_t* iters, uint8_t* pass, cudaStream_t stream, const TraceSpec* tr = nullptr) {
    if (!C) return fail(NGDBF_ERR_INVALID_ARG, "code is NULL");
    ngdbf_status s = check_params(P, sigma);
    if (s != NGDBF_OK) return s;
    if (n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
    g_last_launch = {0, 0, 0, 0, 0, 0};
    if (n_frames == 0) return NGDBF_OK;
    if (!y || !bits || !iters || !pass) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != C->device) return fail(NGDBF_ERR_INVALID_ARG, "code tables belong to another device");
    for (const void* p : {(const void*)y, (const void*)bits, (const void*)iters, (const void*)pass}) {
        cudaPointerAttributes a;
        e = cudaPointerGetAttributes(&a, p);
        if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(NGDBF_ERR_INVALID_ARG, "y, bits, iters and pass must be device memory");
        }
    }
    LaunchPlan plan;
    KernelFn fn;
    int sm_count = 0;
    s = plan_launch(C, P, n_frames, dev, &plan, &fn, &sm_count);
    if (s != NGDBF_OK) return s;

    cudaMemPool_t pool;
    s = get_pool(dev, &pool);
    if (s != NGDBF_OK) return s;
    const bool state = (P->variant & 3) != 0;
    const size_t slot_elems = (size_t)plan.grid * pad4(C->n) * kSlots;
    const size_t bytes_y = (slot_elems * held_bytes(P->precision) + 255) / 256 * 256;
    const size_t bytes_st = (state && !plan.st_smem) ? (slot_elems * 2 + 255) / 256 * 256 : 0;
    const size_t total = 256 + bytes_y + bytes_st;
    void* ws = nullptr;
    e = cudaMallocFromPoolAsync(&ws, total, pool, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NGDBF_ERR_OOM : NGDBF_ERR_CUDA,
                    std::string("scratch allocation: ") + cudaGetErrorString(e));
    }
    unsigned char* base = static_cast<unsigned char*>(ws);

    DecodeArgs A;
    fill_args(C, P, plan, y, n_frames, sigma, seed, frame_offset, bits, iters, pass, base,
              base + 256 + bytes_y, bytes_st != 0, &A);
    if (tr && tr->frames > 0) {
        A.J.trace_u = tr->unsat;
        A.J.trace_c = reinterpret_cast<long long*>(tr->corr);
        A.J.trace_frames = tr->frames;
    }

    e = cudaMemsetAsync(A.J.queue, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess) {
        fn<<<plan.grid, plan.block, plan.smem, stream>>>(A);
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
    set_last_launch(plan.grid, plan.block, plan.smem, plan.st_smem ? 1 : 0, plan.placement, 1, sm_count);
    return NGDBF_OK;
}

}  // namespace host
}  // namespace ngdbf

using namespace ngdbf::host;

extern "C" {

const char* ngdbf_last_error(void) { return g_last_error.c_str(); }

ngdbf_status ngdbf_last_host_stats(ngdbf_host_stats* out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = g_last_host;
    return NGDBF_OK;
}

ngdbf_status ngdbf_last_launch(ngdbf_launch_info* out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = g_last_launch;
    return NGDBF_OK;
}

ngdbf_status ngdbf_code_create(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                               ngdbf_code_t** out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!row_ptr || !col_idx) return fail(NGDBF_ERR_INVALID_ARG, "NULL row_ptr or col_idx");
    if (!(n > m && m >= 1)) return fail(NGDBF_ERR_INVALID_ARG, "need n > m >= 1");
    if (n > NGDBF_MAX_N) return fail(NGDBF_ERR_UNSUPPORTED, "n above NGDBF_MAX_N");
    if (row_ptr[0] != 0) return fail(NGDBF_ERR_INVALID_ARG, "row_ptr[0] must be 0");
    std::vector<int32_t> sdeg(n, 0);
    int dc_max = 0;
    std::vector<int32_t> mark(n, -1);
    for (int i = 0; i < m; ++i) {
        const int d = row_ptr[i + 1] - row_ptr[i];
        if (d < 1) return fail(NGDBF_ERR_INVALID_ARG, "every check needs degree >= 1");
        if (d > NGDBF_MAX_DEGREE) return fail(NGDBF_ERR_UNSUPPORTED, "check degree above NGDBF_MAX_DEGREE");
        dc_max = std::max(dc_max, d);
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int c = col_idx[e];
            if (c < 0 || c >= n) return fail(NGDBF_ERR_INVALID_ARG, "column index out of range");
            if (mark[c] == i) return fail(NGDBF_ERR_INVALID_ARG, "repeated column in a row");
            mark[c] = i;
            sdeg[c] += 1;
        }
    }
    int dv_max = 0;
    for (int k = 0; k < n; ++k) {
        if (sdeg[k] < 1) return fail(NGDBF_ERR_INVALID_ARG, "every symbol needs degree >= 1");
        dv_max = std::max(dv_max, sdeg[k]);
    }
    if (dv_max > NGDBF_MAX_DEGREE) return fail(NGDBF_ERR_UNSUPPORTED, "symbol degree above NGDBF_MAX_DEGREE");
    // N(i) column-major [j][i], padded with the zero-word sentinel n
    std::vector<uint16_t> chk((size_t)dc_max * m, (uint16_t)n);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) chk[(size_t)(e - row_ptr[i]) * m + i] = (uint16_t)col_idx[e];
    // M(k) row-major [k][j], padded with the zero-word sentinel m
    std::vector<uint16_t> sym((size_t)n * dv_max, (uint16_t)m);
    std::vector<uint8_t> deg(n);
    std::vector<int32_t> fill(n, 0);
    for (int i = 0; i < m; ++i)
        for (int e = row_ptr[i]; e < row_ptr[i + 1]; ++e) {
            const int c = col_idx[e];
            sym[(size_t)c * dv_max + fill[c]++] = (uint16_t)i;
        }
    for (int k = 0; k < n; ++k) deg[k] = (uint8_t)sdeg[k];

    ngdbf_code* C = new (std::nothrow) ngdbf_code;
    if (!C) return fail(NGDBF_ERR_OOM, "host allocation");
    C->n = n; C->m = m; C->dv_max = dv_max; C->dc_max = dc_max;
    C->d_chk_cols = nullptr; C->d_sym_chks = nullptr; C->d_sym_deg = nullptr;
    cudaError_t e = cudaGetDevice(&C->device);
    if (e == cudaSuccess) e = cudaMalloc(&C->d_chk_cols, chk.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&C->d_sym_chks, sym.size() * 2);
    if (e == cudaSuccess) e = cudaMalloc(&C->d_sym_deg, deg.size());
    if (e == cudaSuccess) e = cudaMemcpy(C->d_chk_cols, chk.data(), chk.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(C->d_sym_chks, sym.data(), sym.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(C->d_sym_deg, deg.data(), deg.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(C->d_chk_cols); cudaFree(C->d_sym_chks); cudaFree(C->d_sym_deg);
        delete C;
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NGDBF_ERR_OOM : NGDBF_ERR_CUDA,
                    std::string("code tables: ") + cudaGetErrorString(e));
    }
    *out = C;
    return NGDBF_OK;
}

ngdbf_status ngdbf_pool_usage(int32_t reset_high, int64_t* used_now, int64_t* used_high) {
    if (!used_now || !used_high) return fail(NGDBF_ERR_INVALID_ARG, "NULL output");
    *used_now = 0;
    *used_high = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(NGDBF_ERR_UNSUPPORTED, "device index out of range");
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        pool = g_pools[dev];
    }
    if (!pool) return NGDBF_OK;
    uint64_t cur = 0, high = 0;
    e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &cur);
    if (e == cudaSuccess && reset_high) {
        uint64_t zero = 0;              // resets the mark to the current use
        e = cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero);
    }
    if (e == cudaSuccess) e = cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &high);
    if (e != cudaSuccess) return cuda_fail(e, "pool attributes");
    *used_now = (int64_t)cur;
    *used_high = (int64_t)high;
    return NGDBF_OK;
}

ngdbf_status ngdbf_code_destroy(ngdbf_code_t* C) {
    if (!C) return NGDBF_OK;
    cudaFree(C->d_chk_cols);
    cudaFree(C->d_sym_chks);
    cudaFree(C->d_sym_deg);
    delete C;
    return NGDBF_OK;
}

ngdbf_status ngdbf_code_info(const ngdbf_code_t* C, int32_t* n, int32_t* m, int32_t* dv_max, int32_t* dc_max) {
    if (!C) return fail(NGDBF_ERR_INVALID_ARG, "code is NULL");
    if (n) *n = C->n;
    if (m) *m = C->m;
    if (dv_max) *dv_max = C->dv_max;
    if (dc_max) *dc_max = C->dc_max;
    return NGDBF_OK;
}

ngdbf_status ngdbf_decode(const ngdbf_code_t* C, const float* y, int64_t n_frames, float sigma,
                          const ngdbf_params* P, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
                          int32_t* iters, uint8_t* pass, void* stream) {
    return decode_impl(C, y, n_frames, sigma, P, seed, frame_offset, bits, iters, pass,
                       static_cast<cudaStream_t>(stream));
}

ngdbf_status ngdbf_decode_trace(const ngdbf_code_t* C, const float* y, int64_t n_frames, float sigma,
                                const ngdbf_params* P, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
                                int32_t* iters, uint8_t* pass, int64_t trace_frames, int32_t* trace_unsat,
                                int64_t* trace_corr, void* stream) {
    if (!P) return fail(NGDBF_ERR_INVALID_ARG, "params is NULL");
    if (trace_frames < 0 || trace_frames > n_frames) return fail(NGDBF_ERR_INVALID_ARG, "need 0 <= trace_frames <= n_frames");
    if (trace_frames > 0) {
        if (!trace_unsat || !trace_corr) return fail(NGDBF_ERR_INVALID_ARG, "NULL trace buffer");
        if (!(P->y_max > 0.0f && P->y_max < 1073741824.0f))
            return fail(NGDBF_ERR_INVALID_ARG, "the objective trace needs a finite y_max below 2^30");
        for (const void* p : {(const void*)trace_unsat, (const void*)trace_corr}) {
            cudaPointerAttributes a;
            cudaError_t e = cudaPointerGetAttributes(&a, p);
            if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
                cudaGetLastError();
                return fail(NGDBF_ERR_INVALID_ARG, "trace buffers must be device memory");
            }
        }
    }
    const TraceSpec tr = {trace_frames, trace_unsat, trace_corr};
    return decode_impl(C, y, n_frames, sigma, P, seed, frame_offset, bits, iters, pass,
                       static_cast<cudaStream_t>(stream), &tr);
}

ngdbf_status ngdbf_decode_host(const ngdbf_code_t* C, const float* y_host, int64_t n_frames, float sigma,
                               const ngdbf_params* P, uint64_t seed, uint64_t frame_offset,
                               uint8_t* bits_host, int32_t* iters_host, uint8_t* pass_host,
                               int64_t chunk_frames) {
    if (!C) return fail(NGDBF_ERR_INVALID_ARG, "code is NULL");
    ngdbf_status s = check_params(P, sigma);
    if (s != NGDBF_OK) return s;
    if (n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return NGDBF_OK;
    if (!y_host || !bits_host || !iters_host || !pass_host) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    const int64_t n = C->n, nb = (C->n + 7) / 8;
    // chunk sizes: the caller's, or a ramp -- an eighth of a quarter of the call first (so
    // that little copying is exposed before the first decode), doubling up to a quarter of
    // the call (so that only the last chunk's tail, where a CTA waits for its slowest frame,
    // is exposed), chunks between 256 MB and 2 GB of samples and at least 4096 frames
    int64_t first_chunk = chunk_frames;
    if (chunk_frames <= 0) {
        const int64_t lo = std::max<int64_t>(4096, (int64_t)(256ll << 20) / (4 * n));
        const int64_t hi = std::max<int64_t>(lo, (int64_t)(2048ll << 20) / (4 * n));
        chunk_frames = std::min(hi, std::max(lo, (n_frames + 3) / 4));
        first_chunk = std::max<int64_t>(std::min<int64_t>(4096, chunk_frames), chunk_frames / 8);
    }
    chunk_frames = std::min(chunk_frames, n_frames);
    first_chunk = std::min(first_chunk, chunk_frames);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    cudaMemPool_t pool;
    s = get_pool(dev, &pool);
    if (s != NGDBF_OK) return s;
    cudaStream_t st[2] = {nullptr, nullptr};
    void* buf[2] = {nullptr, nullptr};
    auto align256 = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t by = (size_t)chunk_frames * n * 4, bb = (size_t)chunk_frames * nb, bi = (size_t)chunk_frames * 4;
    const size_t bp = (size_t)chunk_frames;
    const size_t per = align256(by) + align256(bb) + align256(bi) + align256(bp);
    ngdbf_status rs = NGDBF_OK;
    g_last_host = ngdbf_host_stats{};
    for (int b = 0; b < 2 && rs == NGDBF_OK; ++b) {
        e = cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&buf[b], per, pool, st[b]);
        if (e != cudaSuccess) rs = cuda_fail(e, "host decode set-up");
    }
    // per chunk: events before the copy in, after it, after the decode and after the copy out
    std::vector<cudaEvent_t> ev;
    auto mark = [&](cudaStream_t s_) {
        cudaEvent_t x = nullptr;
        if (cudaEventCreate(&x) == cudaSuccess) {
            ev.push_back(x);
            cudaEventRecord(x, s_);
        } else {
            cudaGetLastError();
            ev.push_back(nullptr);
        }
    };
    // samples through the library's staging buffers (host threads + copies from reused
    // page-locked memory) unless direct copies were asked for
    Staging* stage = host_copy_mode() == NGDBF_HOST_COPY_STAGED ? staging_acquire(dev) : nullptr;
    int64_t kernels = 0, chunks = 0;
    for (int64_t off = 0, c = 0, size = first_chunk; off < n_frames && rs == NGDBF_OK;
         off += size, size = std::min(2 * size, chunk_frames), ++c) {
        const int b = (int)(c & 1);
        const int64_t F = std::min(size, n_frames - off);
        unsigned char* p = static_cast<unsigned char*>(buf[b]);
        float* dy = reinterpret_cast<float*>(p);
        uint8_t* dbits = p + align256(by);
        int32_t* diters = reinterpret_cast<int32_t*>(dbits + align256(bb));
        uint8_t* dpass = reinterpret_cast<uint8_t*>(diters) + align256(bi);
        mark(st[b]);
        e = stage ? staged_h2d(stage, dy, y_host + off * n, (size_t)F * n * 4, st[b])
                  : cudaMemcpyAsync(dy, y_host + off * n, (size_t)F * n * 4, cudaMemcpyHostToDevice, st[b]);
        if (e != cudaSuccess) { rs = cuda_fail(e, "host-to-device copy"); break; }
        mark(st[b]);
        rs = decode_impl(C, dy, F, sigma, P, seed, frame_offset + (uint64_t)off, dbits, diters, dpass, st[b]);
        if (rs != NGDBF_OK) break;
        kernels += g_last_launch.kernels;
        mark(st[b]);
        e = cudaMemcpyAsync(bits_host + off * nb, dbits, (size_t)F * nb, cudaMemcpyDeviceToHost, st[b]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(iters_host + off, diters, (size_t)F * 4, cudaMemcpyDeviceToHost, st[b]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pass_host + off, dpass, (size_t)F, cudaMemcpyDeviceToHost, st[b]);
        if (e != cudaSuccess) rs = cuda_fail(e, "device-to-host copy");
        mark(st[b]);
        g_last_host.h2d_bytes += (int64_t)F * n * 4;
        g_last_host.d2h_bytes += (int64_t)F * (nb + 5);
        ++chunks;
    }
    for (int b = 0; b < 2; ++b) {
        if (buf[b]) cudaFreeAsync(buf[b], st[b]);
        if (st[b]) {
            cudaError_t es = cudaStreamSynchronize(st[b]);
            if (es != cudaSuccess && rs == NGDBF_OK) rs = cuda_fail(es, "stream synchronize");
            cudaStreamDestroy(st[b]);
        }
    }
    staging_release(stage);     // every copy out of it has completed
    if (rs == NGDBF_OK && chunks > 0 && ev.size() == (size_t)chunks * 4) {
        auto ms = [&](cudaEvent_t a, cudaEvent_t b_) {
            float v = 0.0f;
            if (a && b_ && cudaEventElapsedTime(&v, a, b_) == cudaSuccess) return (double)v;
            cudaGetLastError();
            return 0.0;
        };
        g_last_host.chunks = (int32_t)chunks;
        double first = 0.0, last = 0.0;
        for (int64_t c = 0; c < chunks; ++c) {
            cudaEvent_t* q = ev.data() + 4 * c;
            g_last_host.h2d_ms += ms(q[0], q[1]);
            g_last_host.kernel_ms += ms(q[1], q[2]);
            g_last_host.d2h_ms += ms(q[2], q[3]);
            last = std::max(last, ms(ev[0], q[3]));
            first = std::min(first, ms(ev[0], q[0]));
        }
        g_last_host.wall_ms = last - first;
    }
    for (cudaEvent_t x : ev)
        if (x) cudaEventDestroy(x);
    if (rs == NGDBF_OK) g_last_launch.kernels = (int32_t)kernels;
    return rs;
}

// ---------------------------------------------------------------------------
// ngdbf_decode_noalloc: the same decode with its scratch in a static device
// array instead of pool memory, for callers that cannot allocate.
// ---------------------------------------------------------------------------

}  // extern "C"

namespace {

// Work counter (first 256 bytes), then per-slot samples [grid][n][32] and, when
// the per-slot state does not fit shared memory, the state words [grid][n][32].
static __device__ __align__(256) unsigned char g_noalloc_scratch[NGDBF_NOALLOC_SCRATCH_BYTES];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[64] = {};

// Device address of g_noalloc_scratch on the current device, looked up once per device.
ngdbf_status noalloc_scratch(int dev, unsigned char** out) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 64) return fail(NGDBF_ERR_UNSUPPORTED, "device index out of range");
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) return cuda_fail(e, "cudaGetSymbolAddress(static scratch)");
        g_noalloc_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_noalloc_addr[dev]);
    return NGDBF_OK;
}

}  // namespace

extern "C" ngdbf_status ngdbf_decode_noalloc(const ngdbf_code_t* C, const float* y, int64_t n_frames,
                                             float sigma, const ngdbf_params* P, uint64_t seed,
                                             uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                                             uint8_t* pass, void* stream_ptr) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    if (!C) return fail(NGDBF_ERR_INVALID_ARG, "code is NULL");
    ngdbf_status s = check_params(P, sigma);
    if (s != NGDBF_OK) return s;
    if (n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
    g_last_launch = {0, 0, 0, 0, 0, 0};
    if (n_frames == 0) return NGDBF_OK;
    if (!y || !bits || !iters || !pass) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != C->device) return fail(NGDBF_ERR_INVALID_ARG, "code tables belong to another device");
    for (const void* p : {(const void*)y, (const void*)bits, (const void*)iters, (const void*)pass}) {
        cudaPointerAttributes a;
        e = cudaPointerGetAttributes(&a, p);
        if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(NGDBF_ERR_INVALID_ARG, "y, bits, iters and pass must be device memory");
        }
    }
    unsigned char* base = nullptr;
    s = noalloc_scratch(dev, &base);
    if (s != NGDBF_OK) return s;
    LaunchPlan plan;
    KernelFn fn;
    int sm_count = 0;
    s = plan_launch(C, P, n_frames, dev, &plan, &fn, &sm_count);
    if (s != NGDBF_OK) return s;

    // Fit the launch into the static array: fewer CTAs when a full grid does not fit.
    const bool state = (P->variant & 3) != 0;
    const size_t per_cta_y = (size_t)pad4(C->n) * kSlots * held_bytes(P->precision);
    const size_t per_cta_st = (state && !plan.st_smem) ? (size_t)pad4(C->n) * kSlots * 2 : 0;
    const size_t avail = (size_t)NGDBF_NOALLOC_SCRATCH_BYTES - 256 - 256;   // counter + alignment
    const size_t max_grid = avail / (per_cta_y + per_cta_st);
    if (max_grid < 1)
        return fail(NGDBF_ERR_UNSUPPORTED, "code needs more per-CTA scratch (" +
                    std::to_string(per_cta_y + per_cta_st) + " bytes) than the static array holds (" +
                    std::to_string((long long)NGDBF_NOALLOC_SCRATCH_BYTES) + " bytes)");
    const int grid = (int)std::min<size_t>((size_t)plan.grid, max_grid);
    const size_t bytes_y = ((size_t)grid * per_cta_y + 255) / 256 * 256;

    DecodeArgs A;
    fill_args(C, P, plan, y, n_frames, sigma, seed, frame_offset, bits, iters, pass, base,
              base + 256 + bytes_y, per_cta_st != 0, &A);
    // The work counter must start at zero; the kernel initializes everything else it reads.
    e = cudaMemsetAsync(A.J.queue, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the static work counter");
    fn<<<grid, plan.block, plan.smem, stream>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    set_last_launch(grid, plan.block, plan.smem, plan.st_smem ? 1 : 0, plan.placement, 1, sm_count);
    return NGDBF_OK;
}

// ---------------------------------------------------------------------------
// Job tables: several decode jobs in one persistent launch (ngdbf_multi.cu).
// ---------------------------------------------------------------------------

#include "ngdbf_multi.h"

struct ngdbf_batch {
    int device = 0, n_jobs = 0, sm_count = 0;
    void* fn = nullptr;                 // job-table kernel
    int grid = 0, block = 0, smem = 0, state_in_smem = 0, tables_in_smem = 0, cluster = 1;
    MultiArgs args;
    unsigned char* d_mem = nullptr;     // jobs | thresholds | queues | first_job | samples | state
    unsigned char* d_st = nullptr;      // per-slot state when it is not in shared memory
    unsigned long long* d_queues = nullptr;
    int32_t* d_first = nullptr;
    std::vector<int64_t> frames, weight;
    std::vector<int> n_of_job;
    std::vector<TableShape> shapes;
    int shape = 0;                      // index of the shape in use
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace ngdbf {
namespace host {

// First job of every CTA: CTAs in proportion to the estimated work of each job
// (frames x n x (T + 1)), at least one CTA per job with frames, at most one CTA
// per 32 of its frames; CTAs left over go to the jobs with the most work per CTA.
std::vector<int32_t> assign_ctas(const std::vector<int64_t>& frames, const std::vector<int64_t>& weight, int grid) {
    std::vector<int64_t> cap(frames.size());
    for (size_t j = 0; j < frames.size(); ++j) cap[j] = (frames[j] + kSlots - 1) / kSlots;
    return assign_ctas_capped(frames, weight, cap, grid);
}

// The same with explicit caps (the most CTAs, or clusters, a job can keep busy).
std::vector<int32_t> assign_ctas_capped(const std::vector<int64_t>& frames, const std::vector<int64_t>& weight,
                                        const std::vector<int64_t>& cap, int grid) {
    const int J = (int)frames.size();
    std::vector<int64_t> cnt(J, 0);
    double total = 0;
    for (int j = 0; j < J; ++j) total += (double)weight[j];
    int used = 0;
    for (int j = 0; j < J; ++j) {
        if (frames[j] == 0) continue;
        int64_t c = (int64_t)std::floor((double)grid * (double)weight[j] / std::max(total, 1.0));
        cnt[j] = std::min(std::max<int64_t>(c, 1), cap[j]);
        used += (int)cnt[j];
    }
    while (used > grid) {                       // more jobs than CTAs: trim the lightest loads
        int pick = -1;
        double best = 1e300;
        for (int j = 0; j < J; ++j)
            if (cnt[j] > 1 || (cnt[j] == 1 && used > grid)) {
                const double per = (double)weight[j] / (double)cnt[j];
                if (cnt[j] > 0 && per < best) { best = per; pick = j; }
            }
        if (pick < 0) break;
        cnt[pick] -= 1;
        used -= 1;
    }
    while (used < grid) {
        int pick = -1;
        double best = -1;
        for (int j = 0; j < J; ++j)
            if (cnt[j] < cap[j]) {
                const double per = (double)weight[j] / (double)(cnt[j] + 1);
                if (per > best) { best = per; pick = j; }
            }
        if (pick < 0) break;
        cnt[pick] += 1;
        used += 1;
    }
    std::vector<int32_t> first;
    first.reserve(grid);
    for (int j = 0; j < J; ++j)
        for (int64_t c = 0; c < cnt[j]; ++c) first.push_back(j);
    while ((int)first.size() < grid) first.push_back(-1);   // no frames left to start on
    return first;
}

// Dynamic shared memory of a job-table launch in which every job gets its own layout
// (job_layout, as the kernels evaluate it): the largest job's bytes, each job taking as many
// of the `tables` as fit in `limit`; -1 when some job does not fit at all.  With a cluster of
// C > 1 CTAs, jobs of at least split_min_n symbols hold their share of the symbols per CTA.
int table_smem(const ngdbf_job* jobs, int32_t n_jobs, int C, int split_min_n, bool adapt, bool st, bool wide,
               int tables, int limit) {
    int total = 0;
    for (int j = 0; j < n_jobs; ++j) {
        const ngdbf_code* c = jobs[j].code;
        const int n_local = (C > 1 && c->n >= split_min_n) ? split_local_max(c->n, C) : c->n;
        int tb = 0;
        const SmemLayout L = job_layout(c->n, c->m, jobs[j].params.t_max, c->dv_max, c->dc_max, adapt, st, wide,
                                        tables, n_local, limit, &tb);
        if (L.total > limit) return -1;
        total = std::max(total, L.total);
    }
    return total;
}

ngdbf_status plan_table(const ngdbf_job* jobs, int32_t n_jobs, int dev, TablePlan* out) {
    TablePlan& T = *out;
    T = TablePlan();
    const int variant = jobs[0].params.variant, precision = jobs[0].params.precision;
    for (int j = 0; j < n_jobs; ++j) {
        const ngdbf_job& q = jobs[j];
        if (!q.code) return fail(NGDBF_ERR_INVALID_ARG, "job without a code");
        ngdbf_status s = check_params(&q.params, q.sigma);
        if (s != NGDBF_OK) return s;
        if (q.params.variant != variant || q.params.precision != precision)
            return fail(NGDBF_ERR_UNSUPPORTED, "jobs of one table must share variant and precision");
        if (q.code->device != dev) return fail(NGDBF_ERR_INVALID_ARG, "code tables belong to another device");
        if (q.n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
        T.n_max = std::max(T.n_max, q.code->n);
        T.m_max = std::max(T.m_max, q.code->m);
        T.t_max = std::max(T.t_max, q.params.t_max);
        T.dv_max = std::max(T.dv_max, q.code->dv_max);
        T.dc_max = std::max(T.dc_max, q.code->dc_max);
        T.thr_words += (size_t)q.params.t_max + 1;
    }
    T.variant = variant;
    T.precision = precision;
    int smem_optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&T.sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    // shared memory for the largest code and T; state, then tables, move out when needed
    const bool state = (variant & 3) != 0, adapt = (variant & NGDBF_ADAPT) != 0;
    T.wide = T.dv_max > 7;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, multi_kernel_fn(variant, precision, state, T.wide));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
    const int limit = smem_optin - (int)fa.sharedSizeBytes;
    // the state in shared memory whenever every job fits with it there; then the most resident
    // warps per SM, the most CTAs per SM, more tables in shared memory (as in choose_placement)
    int best_warps = 0, best_bps = 0;
    for (const bool st : {true, false}) {
        if (st && !state) continue;
        if (best_bps > 0) break;
        void* fn = multi_kernel_fn(variant, precision, st, T.wide);
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
        for (const int tb : {kTabChk | kTabSym, kTabChk, 0}) {
            const int total = table_smem(jobs, n_jobs, 1, INT32_MAX, adapt, st, T.wide, tb, limit);
            if (total < 0) continue;
            for (const int block : {1024, 512, 256}) {
                int bps = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)fn, block, total);
                if (e != cudaSuccess) return cuda_fail(e, "occupancy");
                const int warps = bps * block / 32;
                if (bps > 0 && (warps > best_warps || (warps == best_warps && bps > best_bps))) {
                    best_warps = warps;
                    best_bps = bps;
                    T.fn = fn;
                    T.smem = total;
                    T.st_smem = st;
                    T.placement = tb;
                }
            }
        }
    }
    if (best_bps == 0) return fail(NGDBF_ERR_UNSUPPORTED, "code too large for the shared-memory decision words");
    T.state_global = state && !T.st_smem;
    for (int block : {1024, 512, 256}) {
        int bps = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)T.fn, block, T.smem);
        if (e != cudaSuccess) return cuda_fail(e, "occupancy");
        if (bps > 0) T.shapes.push_back({block, bps});
    }
    if (T.shapes.empty()) return fail(NGDBF_ERR_UNSUPPORTED, "job-table kernel does not fit on an SM");
    return NGDBF_OK;
}

// Codes of at least this many symbols are split over the CTAs of a cluster.
constexpr int kSplitMinN = 2048;

ngdbf_status table_shapes(const TablePlan& T, const ngdbf_job* jobs, int32_t n_jobs, int dev,
                          std::vector<TableShape>* out) {
    out->clear();
    for (const auto& sh : T.shapes) {
        TableShape c;
        c.fn = T.fn; c.block = sh.first; c.cluster = 1; c.grid_max = T.sm_count * sh.second; c.smem = T.smem;
        c.placement = T.placement; c.n_local = T.n_max; c.split_min_n = INT32_MAX;
        c.st_smem = T.st_smem; c.state_global = T.state_global;
        out->push_back(c);
    }
    int smem_optin = 0;
    cudaError_t e = cudaDeviceGetAttribute(&smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    const bool state = (T.variant & 3) != 0, adapt = (T.variant & NGDBF_ADAPT) != 0;
    const int variant = T.variant, precision = T.precision;
    const bool wide = T.wide;
    {
        // no cluster, the other placements of the adjacency tables that fit with the plan's state
        cudaFuncAttributes fa;
        e = cudaFuncGetAttributes(&fa, T.fn);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFuncGetAttributes");
        const int limit = smem_optin - (int)fa.sharedSizeBytes;
        for (const int tb : {kTabChk | kTabSym, kTabChk, 0}) {
            if (tb == T.placement) continue;
            const int total = table_smem(jobs, n_jobs, 1, INT32_MAX, adapt, T.st_smem, wide, tb, limit);
            if (total < 0 || total == T.smem) continue;    // no fit, or the same layouts as the plan's
            for (const int block : {1024, 512}) {
                int bps = 0;
                e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, (const void*)T.fn, block, total);
                if (e != cudaSuccess) return cuda_fail(e, "occupancy");
                if (bps <= 0) continue;
                TableShape c;
                c.fn = T.fn; c.block = block; c.cluster = 1; c.grid_max = T.sm_count * bps; c.smem = total;
                c.placement = tb; c.n_local = T.n_max; c.split_min_n = INT32_MAX;
                c.st_smem = T.st_smem; c.state_global = T.state_global;
                out->push_back(c);
            }
        }
    }
    // cluster candidates: codes of at least smin symbols split over the C CTAs of a cluster
    // (smin = kSplitMinN first, so that the candidates' order does not depend on the others;
    // then the other thresholds where they split a different set of codes)
    auto cluster_shapes = [&](int C, int smin) -> ngdbf_status {
        // symbols per CTA: the share of a split code, or a whole code decoded per CTA
        int n_local = 0, n_split = 0;
        for (int j = 0; j < n_jobs; ++j) {
            const int n = jobs[j].code->n;
            if (n >= smin) {
                n_local = std::max(n_local, split_local_max(n, C));
                ++n_split;
            } else {
                n_local = std::max(n_local, n);
            }
        }
        if (n_split == 0) return NGDBF_OK;     // nothing to split
        cudaFuncAttributes fa;
        cudaError_t e2 = cudaFuncGetAttributes(&fa, multi_cluster_kernel_fn(variant, precision, state, wide));
        if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFuncGetAttributes");
        const int limit = smem_optin - (int)fa.sharedSizeBytes;
        for (const bool st : {true, false}) {
            if (st && !state) continue;
            void* fn = multi_cluster_kernel_fn(variant, precision, st, wide);
            e2 = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
            if (e2 != cudaSuccess) return cuda_fail(e2, "cudaFuncSetAttribute");
            bool any = false;
            int prev = -1;
            for (const int tb : {kTabChk | kTabSym, kTabChk, 0}) {
                const int total = table_smem(jobs, n_jobs, C, smin, adapt, st, wide, tb, limit);
                if (total < 0 || total == prev) continue;    // no fit, or the same layouts again
                prev = total;
                for (const int block : {1024, 512}) {
                    const int clusters = max_active_clusters(fn, C, block, total);
                    if (clusters <= 0) continue;
                    TableShape c;
                    c.fn = fn; c.block = block; c.cluster = C; c.grid_max = clusters * C; c.smem = total;
                    c.placement = tb; c.n_local = n_local; c.split_min_n = smin;
                    c.st_smem = st; c.state_global = state && !st;
                    out->push_back(c);
                    any = true;
                }
            }
            if (any) break;                  // the state fits shared memory: keep it there
        }
        return NGDBF_OK;
    };
    auto split_set = [&](int smin) {
        std::vector<bool> v(n_jobs);
        for (int j = 0; j < n_jobs; ++j) v[j] = jobs[j].code->n >= smin;
        return v;
    };
    for (const int C : {2, 4, 8}) {
        ngdbf_status s = cluster_shapes(C, kSplitMinN);
        if (s != NGDBF_OK) return s;
    }
    for (const int smin : {1024, 4096}) {
        if (split_set(smin) == split_set(kSplitMinN)) continue;
        for (const int C : {2, 4, 8}) {
            ngdbf_status s = cluster_shapes(C, smin);
            if (s != NGDBF_OK) return s;
        }
    }
    return NGDBF_OK;
}

}  // namespace host
}  // namespace ngdbf

namespace {

cudaError_t batch_enqueue(ngdbf_batch* B, cudaStream_t stream) {
    cudaError_t e = cudaMemsetAsync(B->d_queues, 0, sizeof(unsigned long long) * B->n_jobs, stream);
    if (e != cudaSuccess) return e;
    return launch_multi(B->fn, B->args, B->grid, B->block, B->smem, stream);
}

// Puts candidate `k` in use: kernel, launch shape, shared-memory plan and the first job of
// every CTA (of every cluster: a split job keeps one cluster busy per 32 frames, a job decoded
// CTA by CTA one cluster per 32 C frames).
ngdbf_status batch_set_shape(ngdbf_batch* B, int k) {
    const TableShape& sh = B->shapes[k];
    const int C = sh.cluster;
    B->shape = k;
    B->fn = sh.fn;
    B->block = sh.block;
    B->smem = sh.smem;
    B->cluster = C;
    B->state_in_smem = sh.st_smem ? 1 : 0;
    B->tables_in_smem = sh.placement;
    B->args.placement = sh.placement;
    B->args.cluster = C;
    B->args.split_min_n = sh.split_min_n;
    B->args.n_local = sh.n_local;
    B->args.smem_bytes = sh.smem;
    B->args.st_global = sh.state_global ? reinterpret_cast<uint16_t*>(B->d_st) : nullptr;
    std::vector<int64_t> cap(B->n_jobs);
    int64_t clusters = 0;
    for (int j = 0; j < B->n_jobs; ++j) {
        const int64_t per = (int64_t)kSlots * (B->n_of_job[j] >= sh.split_min_n ? 1 : C);
        cap[j] = (B->frames[j] + per - 1) / per;
        clusters += cap[j];
    }
    const int64_t n_cl = std::max<int64_t>(1, std::min<int64_t>(sh.grid_max / C, clusters));
    B->grid = (int)(n_cl * C);
    std::vector<int32_t> first = assign_ctas_capped(B->frames, B->weight, cap, (int)n_cl);
    cudaError_t e = cudaMemcpy(B->d_first, first.data(), first.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(e, "job table: first jobs");
    return NGDBF_OK;
}

// Captures queue reset + kernel in a CUDA graph that ngdbf_batch_launch replays.
ngdbf_status batch_capture(ngdbf_batch* B) {
    cudaStream_t cs;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaError_t le = batch_enqueue(B, cs);
        e = cudaStreamEndCapture(cs, &B->graph);
        if (le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, B->graph, 0);
    cudaStreamDestroy(cs);
    if (e != cudaSuccess) return cuda_fail(e, "graph capture of the job table");
    return NGDBF_OK;
}

void batch_free(ngdbf_batch* B) {
    if (!B) return;
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    if (B->d_mem) cudaFree(B->d_mem);
    delete B;
}

}  // namespace

extern "C" ngdbf_status ngdbf_batch_create(const ngdbf_job* jobs, int32_t n_jobs, uint64_t seed, int32_t flags,
                                           void* stream_ptr, ngdbf_batch_t** out) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!jobs || n_jobs < 1) return fail(NGDBF_ERR_INVALID_ARG, "need at least one job");
    if (flags & ~(NGDBF_BATCH_TUNE | NGDBF_BATCH_GRAPH)) return fail(NGDBF_ERR_INVALID_ARG, "unknown flags");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    TablePlan T;
    ngdbf_status ps = plan_table(jobs, n_jobs, dev, &T);
    if (ps != NGDBF_OK) return ps;
    for (int j = 0; j < n_jobs; ++j) {
        const ngdbf_job& q = jobs[j];
        if (q.n_frames == 0) continue;
        if (!q.y || !q.bits || !q.iters || !q.pass) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
        for (const void* p : {(const void*)q.y, (const void*)q.bits, (const void*)q.iters, (const void*)q.pass}) {
            cudaPointerAttributes a;
            e = cudaPointerGetAttributes(&a, p);
            if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
                cudaGetLastError();
                return fail(NGDBF_ERR_INVALID_ARG, "job buffers must be device memory");
            }
        }
    }
    ngdbf_batch* B = new (std::nothrow) ngdbf_batch;
    if (!B) return fail(NGDBF_ERR_OOM, "host allocation");
    B->device = dev;
    B->n_jobs = n_jobs;
    B->sm_count = T.sm_count;
    ngdbf_status ss = table_shapes(T, jobs, n_jobs, dev, &B->shapes);
    if (ss != NGDBF_OK) { batch_free(B); return ss; }
    // scratch for the largest candidate: per CTA the samples (and state) of its symbols
    size_t grid_max = 0, bytes_y = 0, bytes_st = 0;
    for (const TableShape& sh : B->shapes) {
        grid_max = std::max(grid_max, (size_t)sh.grid_max);
        bytes_y = std::max(bytes_y, (size_t)sh.grid_max * pad4(sh.n_local) * kSlots * held_bytes(T.precision));
        if (sh.state_global) bytes_st = std::max(bytes_st, (size_t)sh.grid_max * pad4(sh.n_local) * kSlots * 2);
    }
    const size_t off_jobs = 0, off_thr = align256(sizeof(Job) * n_jobs), off_q = off_thr + align256(T.thr_words * 4);
    const size_t off_first = off_q + align256(8 * (size_t)n_jobs), off_y = off_first + align256(4 * grid_max);
    const size_t off_st = off_y + align256(bytes_y);
    const size_t total = off_st + align256(bytes_st);
    e = cudaMalloc(&B->d_mem, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        batch_free(B);
        return fail(e == cudaErrorMemoryAllocation ? NGDBF_ERR_OOM : NGDBF_ERR_CUDA, "job table scratch");
    }
    B->d_queues = reinterpret_cast<unsigned long long*>(B->d_mem + off_q);
    B->d_first = reinterpret_cast<int32_t*>(B->d_mem + off_first);
    B->d_st = bytes_st ? B->d_mem + off_st : nullptr;
    // job table and thresholds
    std::vector<Job> hjobs(n_jobs);
    std::vector<uint32_t> hthr(T.thr_words);
    size_t tpos = 0;
    B->frames.resize(n_jobs);
    B->weight.resize(n_jobs);
    B->n_of_job.resize(n_jobs);
    for (int j = 0; j < n_jobs; ++j) {
        const ngdbf_job& q = jobs[j];
        fill_job(q.code, &q.params, q.y, q.n_frames, q.sigma, q.frame_offset, q.bits, q.iters, q.pass,
                 B->d_queues + j, &hjobs[j], hthr.data() + tpos);
        hjobs[j].thr = reinterpret_cast<const uint32_t*>(B->d_mem + off_thr) + tpos;
        tpos += (size_t)q.params.t_max + 1;
        B->frames[j] = q.n_frames;
        B->weight[j] = q.n_frames * (int64_t)q.code->n * (q.params.t_max + 1);
        B->n_of_job[j] = q.code->n;
    }
    e = cudaMemcpy(B->d_mem + off_jobs, hjobs.data(), sizeof(Job) * n_jobs, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(B->d_mem + off_thr, hthr.data(), hthr.size() * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) { batch_free(B); return cuda_fail(e, "job table upload"); }
    MultiArgs& A = B->args;
    std::memset(&A, 0, sizeof(A));
    A.jobs = reinterpret_cast<const Job*>(B->d_mem + off_jobs);
    A.n_jobs = n_jobs;
    A.first_job = B->d_first;
    A.n_max = T.n_max; A.m_max = T.m_max; A.t_max = T.t_max; A.dv_max = T.dv_max; A.dc_max = T.dc_max;
    A.yslots = B->d_mem + off_y;
    host_gen_consts(seed, A.G);
    // launch shape: the default, or the fastest candidate on this table (block size x cluster
    // size x placement of the adjacency tables)
    ngdbf_status s = batch_set_shape(B, 0);
    if (s == NGDBF_OK && (flags & NGDBF_BATCH_TUNE) && B->shapes.size() > 1) {
        cudaEvent_t t0, t1;
        cudaEventCreate(&t0);
        cudaEventCreate(&t1);
        float best = 1e30f;
        int best_shape = 0;
        for (int k = 0; k < (int)B->shapes.size(); ++k) {
            s = batch_set_shape(B, k);
            if (s != NGDBF_OK) break;
            e = batch_enqueue(B, stream);                    // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(t0, stream);
            if (e == cudaSuccess) e = batch_enqueue(B, stream);
            if (e == cudaSuccess) e = cudaEventRecord(t1, stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(t1);
            if (e != cudaSuccess) { s = cuda_fail(e, "tuning launch"); break; }
            float ms = 0;
            cudaEventElapsedTime(&ms, t0, t1);
            if (ms < best) { best = ms; best_shape = k; }
        }
        cudaEventDestroy(t0);
        cudaEventDestroy(t1);
        if (s == NGDBF_OK) s = batch_set_shape(B, best_shape);
    }
    if (s != NGDBF_OK) { batch_free(B); return s; }
    if (flags & NGDBF_BATCH_GRAPH) {
        s = batch_capture(B);
        if (s != NGDBF_OK) { batch_free(B); return s; }
    }
    *out = B;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_batch_shape(const ngdbf_batch_t* B, int32_t k, int32_t* count, ngdbf_launch_info* info) {
    if (!B) return fail(NGDBF_ERR_INVALID_ARG, "batch is NULL");
    if (count) *count = (int32_t)B->shapes.size();
    if (!info) return NGDBF_OK;
    if (k < 0) k = B->shape;
    if (k >= (int32_t)B->shapes.size()) return fail(NGDBF_ERR_INVALID_ARG, "no such shape");
    const TableShape& sh = B->shapes[k];
    std::memset(info, 0, sizeof(*info));
    info->grid = sh.grid_max;
    info->block = sh.block;
    info->smem_bytes = sh.smem;
    info->state_in_smem = sh.st_smem ? 1 : 0;
    info->kernels = 1;
    info->sm_count = B->sm_count;
    info->tables_in_smem = sh.placement;
    info->cluster = sh.cluster;
    info->split_min_n = sh.cluster > 1 ? sh.split_min_n : 0;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_batch_use_shape(ngdbf_batch_t* B, int32_t k) {
    if (!B) return fail(NGDBF_ERR_INVALID_ARG, "batch is NULL");
    if (k < 0 || k >= (int32_t)B->shapes.size()) return fail(NGDBF_ERR_INVALID_ARG, "no such shape");
    const bool graph = B->exec != nullptr;
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    ngdbf_status s = batch_set_shape(B, k);
    if (s == NGDBF_OK && graph) s = batch_capture(B);
    return s;
}

extern "C" ngdbf_status ngdbf_batch_launch(ngdbf_batch_t* B, void* stream_ptr) {
    if (!B) return fail(NGDBF_ERR_INVALID_ARG, "batch is NULL");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev != B->device) return fail(NGDBF_ERR_INVALID_ARG, "batch belongs to another device");
    e = B->exec ? cudaGraphLaunch(B->exec, stream) : batch_enqueue(B, stream);
    if (e != cudaSuccess) return cuda_fail(e, "job table launch");
    set_last_launch(B->grid, B->block, B->smem, B->state_in_smem, B->tables_in_smem, 1, B->sm_count);
    g_last_launch.cluster = B->cluster;
    g_last_launch.split_min_n = B->cluster > 1 ? B->args.split_min_n : 0;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_batch_destroy(ngdbf_batch_t* B) {
    batch_free(B);
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_generator_table(float* out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    std::memcpy(out, icdf_table().words(), 256 * sizeof(float4));
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_mix_probe(int32_t groups, uint32_t* sink, int64_t* threads_out, void* stream) {
    if (groups < 1 || !sink || !threads_out) return fail(NGDBF_ERR_INVALID_ARG, "need groups >= 1, sink and threads_out");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, sink);
    if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(NGDBF_ERR_INVALID_ARG, "sink must be device memory");
    }
    int dev = 0, sms = 0, bps = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, mix_probe_kernel, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e, "probe set-up");
    GenConsts G;
    host_gen_consts(3, G);
    const int grid = sms * std::max(bps, 1);
    mix_probe_kernel<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(G, groups, sink);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "probe launch");
    *threads_out = (int64_t)grid * 256;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_gaussian_range(uint32_t start, uint32_t count, float* z, void* stream) {
    if (count == 0) return NGDBF_OK;
    if (!z) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, z);
    if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
        cudaGetLastError();
        return fail(NGDBF_ERR_INVALID_ARG, "z must be device memory");
    }
    GenConsts G;
    host_gen_consts(0, G);
    const uint32_t blocks = std::min<uint32_t>((count + 255) / 256, 152u * 64u);
    gaussian_range_kernel<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(G, start, count, z);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gaussian range");
    return NGDBF_OK;
}
