// ngdbf_decode.cu -- persistent slot-refill NGDBF decoder for sm_103a and its C ABI.
//
// Work decomposition.  A CTA owns 32 frame slots, one per bit of a 32-bit
// word: the decisions x_k of its 32 frames are one word per symbol k and the
// syndromes s_i one word per check i (bit f set <=> x_k = -1 / check i
// unsatisfied for slot f).  Each round the CTA
//   A. forms every syndrome word as the XOR of the d_c decision words of a
//      check (Sec. III-A, Step 1 of Sec. III-B), OR-reduces them to the
//      "some check unsatisfied" mask with warp reductions,
//   B. retires slots whose frame satisfied every check (pass) or reached T
//      (smoothed output, Sec. III-E), writes their outputs, takes new frames
//      from a global atomic queue for them and loads those frames, then
//   C. runs Step 2 / Step 3b for every symbol of every live slot: a warp
//      processes four symbols (one Philox call) at a time with lane = slot,
//      counts the lane's unsatisfied checks among M(k), forms
//      E_k = x_k y_k + w S_k + q_k, compares it with theta lambda^{u_k},
//      adapts u_k, accumulates the smoothing counter, and rebuilds the
//      decision word with a warp ballot.
// Slots therefore iterate independently (each frame has its own t), a
// converged frame frees its slot at once, and the CTA only stops when the
// queue is empty and its last slot finished.
//
// Per-(symbol, slot) state: the saturated sample (FP32, global scratch laid
// out [k][slot], L2-resident), and a 16-bit word holding u_k (bits 0-8) and
// the number of -1 decisions inside the smoothing window (bits 9-15), in
// shared memory when it fits, else in global scratch.  Decision and syndrome
// words, the code adjacency, and the threshold table live in shared memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/ngdbf.h"
#include "ngdbf_device.cuh"

namespace ngdbf {

constexpr int kSlots = 32;
constexpr int kMaxT = NGDBF_MAX_T;
constexpr uint32_t kUMask = 0x1FFu;   // u_k: bits 0-8
constexpr int kCShift = 9;            // smoothing count: bits 9-15

struct DecodeArgs {
    // code tables (device)
    int32_t n, m, dv_max, dc_max;
    const uint16_t* chk_cols;   // [dc_max][m]   N(i) column-major, padded with n
    const uint16_t* sym_chks;   // [n][dv_max]   M(k) row-major, padded with m
    const uint8_t* sym_deg;     // [n]           d_v(k)
    int32_t tables_smem;        // copy the tables into shared memory
    // batch
    const float* y;             // [n_frames][n]
    int64_t n_frames;
    uint64_t frame_offset;
    uint8_t* bits;              // [n_frames][nb]
    int32_t* iters;
    uint8_t* pass;
    int32_t nb;
    // parameters
    float w, theta, scale, y_max;
    int32_t clamp, t_max, t_smooth;   // t_smooth = max(0, T - W)
    // scratch
    float* yslots;              // [grid][n][32]
    uint16_t* st_global;        // [grid][n][32] when the state is not in shared memory
    unsigned long long* queue;  // next unclaimed frame index
    GenConsts G;
    float thr[kMaxT + 1];       // fl32(theta lambda^u), u = 0..T
};

struct SmemLayout {
    int32_t off_frame, off_start, off_ctl, off_xw, off_sw, off_cnt, off_thr, off_st, off_chk, off_sym, total;
};

// Offsets in bytes of the shared-memory arrays.  ctl holds: [0..1] unsatisfied
// masks (double-buffered by pass parity), [2] live mask, [3] new-slot mask.
// cnt holds per symbol the bit-sliced count of unsatisfied checks (one word per
// count bit, bit f for slot f) and d_v(k): 3 slices + degree in 16 bytes when
// d_v <= 7 (narrow), 7 slices + degree in 32 bytes otherwise (wide).
__host__ __device__ inline SmemLayout smem_layout(int n, int m, int t_max, int dv_max, int dc_max,
                                                  bool need_thr, bool st_smem, bool tables_smem) {
    SmemLayout L;
    int o = 0;
    auto take = [&](int bytes, int align) {
        o = (o + align - 1) / align * align;
        int r = o;
        o += bytes;
        return r;
    };
    const int cnt_bytes = dv_max <= 7 ? 16 : 32;
    L.off_frame = take(kSlots * 8, 16);
    L.off_start = take(kSlots * 4, 16);
    L.off_ctl = take(8 * 4, 16);
    L.off_cnt = take(n * cnt_bytes, 16);
    L.off_xw = take((n + 1) * 4, 16);
    L.off_sw = take((m + 1) * 4, 16);
    L.off_thr = need_thr ? take((t_max + 1) * 4, 16) : -1;
    L.off_st = st_smem ? take(n * kSlots * 2, 16) : -1;
    L.off_chk = tables_smem ? take(dc_max * m * 2, 16) : -1;
    L.off_sym = tables_smem ? take(n * dv_max * 2 + n, 16) : -1;
    L.total = (o + 15) / 16 * 16;
    return L;
}

// Position of the (j+1)-th set bit of mask (j < popc(mask)).
__device__ __forceinline__ int nth_set_bit(uint32_t mask, int j) {
    for (int i = 0; i < j; ++i) mask &= mask - 1u;
    return __ffs(mask) - 1;
}

template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE>
__global__ void __launch_bounds__(1024) ngdbf_persistent_kernel(const __grid_constant__ DecodeArgs A) {
    constexpr bool kState = ADAPT || SMOOTH;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = A.n, m = A.m, T = A.t_max, dv_max = A.dv_max, dc_max = A.dc_max;
    const SmemLayout L = smem_layout(n, m, T, dv_max, dc_max, ADAPT, ST_SMEM && kState, A.tables_smem != 0);
    long long* lane_frame = reinterpret_cast<long long*>(smem + L.off_frame);
    int32_t* lane_start = reinterpret_cast<int32_t*>(smem + L.off_start);
    uint32_t* ctl = reinterpret_cast<uint32_t*>(smem + L.off_ctl);
    uint4* cnt = reinterpret_cast<uint4*>(smem + L.off_cnt);
    uint32_t* xw = reinterpret_cast<uint32_t*>(smem + L.off_xw);
    uint32_t* sw = reinterpret_cast<uint32_t*>(smem + L.off_sw);
    float* thr = ADAPT ? reinterpret_cast<float*>(smem + L.off_thr) : nullptr;
    uint16_t* st = nullptr;
    if constexpr (kState) {
        st = ST_SMEM ? reinterpret_cast<uint16_t*>(smem + L.off_st)
                     : A.st_global + (size_t)blockIdx.x * n * kSlots;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    // adjacency tables: only phases A and A' read them, so a generic pointer to
    // shared or global memory serves both placements
    const uint16_t* chk_cols = A.chk_cols;
    const uint16_t* sym_chks = A.sym_chks;
    const uint8_t* sym_deg = A.sym_deg;
    if (A.tables_smem) {
        uint16_t* c = reinterpret_cast<uint16_t*>(smem + L.off_chk);
        uint16_t* s = reinterpret_cast<uint16_t*>(smem + L.off_sym);
        uint8_t* d = reinterpret_cast<uint8_t*>(s + n * dv_max);
        for (int i = tid; i < dc_max * m; i += blockDim.x) c[i] = A.chk_cols[i];
        for (int i = tid; i < n * dv_max; i += blockDim.x) s[i] = A.sym_chks[i];
        for (int i = tid; i < n; i += blockDim.x) d[i] = A.sym_deg[i];
        chk_cols = c;
        sym_chks = s;
        sym_deg = d;
    }
    float* ys = A.yslots + (size_t)blockIdx.x * n * kSlots;

    // ---- set-up: zero the state, sentinels, thresholds, first 32 frames ----
    for (int k = tid; k <= n; k += blockDim.x) xw[k] = 0u;
    for (int i = tid; i <= m; i += blockDim.x) sw[i] = 0u;
    if constexpr (ADAPT)
        for (int u = tid; u <= T; u += blockDim.x) thr[u] = A.thr[u];
    if constexpr (kState)
        for (int e = tid; e < n * kSlots; e += blockDim.x) st[e] = 0;
    if (tid == 0) {
        for (int c = 0; c < 8; ++c) ctl[c] = 0u;
        const unsigned long long base = atomicAdd(A.queue, (unsigned long long)kSlots);
        uint32_t live = 0;
        for (int f = 0; f < kSlots; ++f) {
            const unsigned long long fid = base + f;
            lane_start[f] = 0;
            if (fid < (unsigned long long)A.n_frames) {
                lane_frame[f] = (long long)fid;
                live |= 1u << f;
            } else {
                lane_frame[f] = -1;
            }
        }
        ctl[2] = live;
        ctl[3] = live;
    }
    __syncthreads();

    int round = 0;   // flip phases executed by this CTA; slot f is at t = round - lane_start[f]
    int pass_id = 0;
    bool refill = true;
    for (;;) {
        if (refill) {
            // ---- load new frames: saturated samples into the slot columns, x(0) = sign(y) ----
            const uint32_t fresh = ctl[3];
            for (int k = tid; k < n; k += blockDim.x) {
                uint32_t word = xw[k] & ~fresh;
                uint32_t rest = fresh;
                while (rest) {
                    const int f = __ffs(rest) - 1;
                    rest &= rest - 1;
                    float v = __ldg(A.y + (size_t)lane_frame[f] * n + k);
                    if (A.clamp) {
                        if (v > A.y_max) v = A.y_max;
                        if (v < -A.y_max) v = -A.y_max;
                    }
                    ys[k * kSlots + f] = v;
                    if (!(v >= 0.0f)) word |= 1u << f;
                    if constexpr (kState) st[k * kSlots + f] = 0;
                }
                xw[k] = word;
            }
            __syncthreads();
            refill = false;
        }

        // ---- A. syndromes (four threads XOR a quarter of a check each) and the vote ----
        {
            uint32_t* unsat = ctl + (pass_id & 1);
            if (tid == 0) ctl[(pass_id + 1) & 1] = 0u;
            uint32_t acc = 0;
            const int per_pass = blockDim.x >> 2, sub = tid & 3;
            for (int base = 0; base < m; base += per_pass) {
                const int i = base + (tid >> 2);
                uint32_t s = 0;
                if (i < m)
                    for (int j = sub; j < dc_max; j += 4) s ^= xw[chk_cols[j * m + i]];
                s ^= __shfl_xor_sync(0xFFFFFFFFu, s, 1);
                s ^= __shfl_xor_sync(0xFFFFFFFFu, s, 2);
                if (i < m && sub == 0) sw[i] = s;
                acc |= s;
            }
            acc = __reduce_or_sync(0xFFFFFFFFu, acc);
            if (lane == 0 && acc) atomicOr(unsat, acc);
            __syncthreads();
        }
        const uint32_t unsat = ctl[pass_id & 1];
        ++pass_id;
        uint32_t live = ctl[2];
        const uint32_t conv = live & ~unsat;
        const int my_t = round - lane_start[lane];
        const uint32_t at_T = __ballot_sync(0xFFFFFFFFu, ((live >> lane) & 1u) && my_t >= T);
        const uint32_t fin = conv | (live & at_T);

        if (fin) {
            // ---- B. outputs of finished slots ----
            const int nfin = __popc(fin);
            const int work = nfin * A.nb;
            for (int idx = tid; idx < work; idx += blockDim.x) {
                const int j = idx / A.nb, b = idx - j * A.nb;
                const int f = nth_set_bit(fin, j);
                const bool ok = (conv >> f) & 1u;
                const int tf = round - lane_start[f];
                uint32_t byte = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int k = 8 * b + q;
                    if (k < n) {
                        uint32_t bit = (xw[k] >> f) & 1u;
                        if constexpr (SMOOTH) {
                            if (!ok) {
                                // X_k = terms - 2 * (#-1 decisions), x(T) included here
                                const int terms = tf - A.t_smooth + 1;
                                const int neg = (int)(st[k * kSlots + f] >> kCShift) + (int)bit;
                                const int X = terms - 2 * neg;
                                bit = X < 0 ? 1u : (X > 0 ? 0u : bit);
                            }
                        }
                        byte |= bit << q;
                    }
                }
                A.bits[(size_t)lane_frame[f] * A.nb + b] = (uint8_t)byte;
            }
            if (tid < nfin) {
                const int f = nth_set_bit(fin, tid);
                const bool ok = (conv >> f) & 1u;
                const long long fr = lane_frame[f];
                A.iters[fr] = ok ? round - lane_start[f] : T;
                A.pass[fr] = ok ? 1 : 0;
            }
            __syncthreads();
            // ---- claim new frames for the finished slots ----
            if (tid == 0) {
                uint32_t fresh = 0;
                const unsigned long long base = atomicAdd(A.queue, (unsigned long long)nfin);
                for (int j = 0; j < nfin; ++j) {
                    const int f = nth_set_bit(fin, j);
                    const unsigned long long fid = base + j;
                    if (fid < (unsigned long long)A.n_frames) {
                        lane_frame[f] = (long long)fid;
                        lane_start[f] = round;
                        fresh |= 1u << f;
                    } else {
                        lane_frame[f] = -1;
                    }
                }
                ctl[2] = (live & ~fin) | fresh;
                ctl[3] = fresh;
            }
            __syncthreads();
            live = ctl[2];
            if (ctl[3]) {
                refill = true;      // new frames need their t = 0 syndrome test first
                continue;
            }
        }
        if (live == 0) break;

        // ---- A'. per symbol, the bit-sliced count of unsatisfied checks in M(k) ----
        for (int k = tid; k < n; k += blockDim.x) {
            const uint16_t* row = sym_chks + k * dv_max;
            if constexpr (!WIDE) {
                uint32_t b0 = 0, b1 = 0, b2 = 0;           // count <= 7: three slices
                for (int e = 0; e < dv_max; ++e) {
                    const uint32_t s = sw[row[e]];
                    const uint32_t c0 = b0 & s;
                    b0 ^= s;
                    const uint32_t c1 = b1 & c0;
                    b1 ^= c0;
                    b2 ^= c1;
                }
                cnt[k] = make_uint4(b0, b1, b2, (uint32_t)sym_deg[k]);
            } else {
                uint32_t b[7] = {0, 0, 0, 0, 0, 0, 0};     // count <= 127: seven slices
                for (int e = 0; e < dv_max; ++e) {
                    uint32_t carry = sw[row[e]];
#pragma unroll
                    for (int q = 0; q < 7; ++q) {
                        const uint32_t c = b[q] & carry;
                        b[q] ^= carry;
                        carry = c;
                    }
                }
                cnt[2 * k] = make_uint4(b[0], b[1], b[2], b[3]);
                cnt[2 * k + 1] = make_uint4(b[4], b[5], b[6], (uint32_t)sym_deg[k]);
            }
        }
        __syncthreads();

        // ---- C. Step 2 and Step 3b for every symbol of every live slot ----
        {
            const bool act = (live >> lane) & 1u;
            const long long fr = lane_frame[lane];
            const uint64_t fid = A.frame_offset + (uint64_t)(act ? fr : 0);
            const uint32_t flo = (uint32_t)fid, fhi = (uint32_t)(fid >> 32);
            const int t = act ? round - lane_start[lane] : 0;
            const bool window = SMOOTH && act && t >= A.t_smooth;
            const int groups = (n + 3) >> 2;
            for (int g = warp; g < groups; g += nwarps) {
                const int k0 = 4 * g;
                // issue the sample and state loads before the generator's arithmetic
                float yv[4];
                uint32_t sv[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const bool in = k0 + j < n;
                    yv[j] = in ? ys[(k0 + j) * kSlots + lane] : 0.0f;
                    if constexpr (kState) sv[j] = in ? (uint32_t)st[(k0 + j) * kSlots + lane] : 0u;
                }
                float z[4];
                gauss4((uint32_t)g, (uint32_t)t, flo, fhi, A.G, z);
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = k0 + j;
                    if (k >= n) break;
                    int unsat_cnt, deg;
                    if constexpr (!WIDE) {
                        const uint4 c = cnt[k];
                        unsat_cnt = (int)(((c.x >> lane) & 1u) | (((c.y >> lane) & 1u) << 1) |
                                          (((c.z >> lane) & 1u) << 2));
                        deg = (int)c.w;
                    } else {
                        const uint4 c = cnt[2 * k], d = cnt[2 * k + 1];
                        unsat_cnt = (int)(((c.x >> lane) & 1u) | (((c.y >> lane) & 1u) << 1) |
                                          (((c.z >> lane) & 1u) << 2) | (((c.w >> lane) & 1u) << 3) |
                                          (((d.x >> lane) & 1u) << 4) | (((d.y >> lane) & 1u) << 5) |
                                          (((d.z >> lane) & 1u) << 6));
                        deg = (int)d.w;
                    }
                    const int S = deg - 2 * unsat_cnt;
                    const uint32_t xword = xw[k];
                    const bool xneg = (xword >> lane) & 1u;
                    const float q = __fmul_rn(A.scale, z[j]);
                    const float E = inversion_metric(xneg, yv[j], S, A.w, q);
                    bool flip;
                    if constexpr (kState) {
                        const uint32_t s0 = sv[j];
                        // u_k <= t - 1 < T for a live slot (cleared on every refill)
                        const float th = ADAPT ? thr[s0 & kUMask] : A.theta;
                        flip = act && (E < th);
                        const uint32_t nv = s0 + ((ADAPT && act && !flip) ? 1u : 0u) +
                                            ((window && xneg) ? (1u << kCShift) : 0u);
                        if (nv != s0) st[k * kSlots + lane] = (uint16_t)nv;
                    } else {
                        flip = act && (E < A.theta);
                    }
                    const uint32_t fm = __ballot_sync(0xFFFFFFFFu, flip);
                    if (lane == 0 && fm) xw[k] = xword ^ fm;
                }
            }
        }
        __syncthreads();
        ++round;
    }
}

}  // namespace ngdbf

// ===========================================================================
// Host side: validation, code tables, launch configuration, C ABI
// ===========================================================================

using namespace ngdbf;

struct ngdbf_code {
    int32_t n, m, dv_max, dc_max;
    int device;
    uint16_t* d_chk_cols;
    uint16_t* d_sym_chks;
    uint8_t* d_sym_deg;
};

namespace {

thread_local std::string g_last_error;
thread_local ngdbf_launch_info g_last_launch = {0, 0, 0, 0, 0, 0};

ngdbf_status fail(ngdbf_status s, const std::string& msg) {
    g_last_error = msg;
    return s;
}

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

void host_gen_consts(uint64_t seed, GenConsts& G) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        G.rk0[r] = k0;
        G.rk1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    for (int j = 1; j <= 5; ++j) G.atanh_c[j - 1] = 1.0f / (float)(2 * j + 1);
    // (pi/2)^n / n! in double by t_n = (t_{n-1} * (pi/2)) / n, then rounded to FP32
    const double half_pi = 1.5707963267948966;
    double t = 1.0;
    for (int nn = 1; nn <= 12; ++nn) {
        t = (t * half_pi) / (double)nn;
        if (nn & 1) {
            const int j = (nn - 1) / 2;
            G.sin_c[j] = (float)((j & 1) ? -t : t);
        } else {
            const int j = nn / 2;
            G.cos_c[j - 1] = (float)((j & 1) ? -t : t);
        }
    }
}

struct LaunchPlan {
    int block, grid, blocks_per_sm, smem;
    bool st_smem, tables_smem;
};

using KernelFn = void (*)(DecodeArgs);

template <bool AD, bool SM>
KernelFn pick_width(bool st_smem, bool wide) {
    if (st_smem) return wide ? ngdbf_persistent_kernel<AD, SM, true, true> : ngdbf_persistent_kernel<AD, SM, true, false>;
    return wide ? ngdbf_persistent_kernel<AD, SM, false, true> : ngdbf_persistent_kernel<AD, SM, false, false>;
}

KernelFn pick_kernel(int variant, bool st_smem, bool wide) {
    switch (variant & 3) {
        case 0: return pick_width<false, false>(st_smem, wide);
        case 1: return pick_width<true, false>(st_smem, wide);
        case 2: return pick_width<false, true>(st_smem, wide);
        default: return pick_width<true, true>(st_smem, wide);
    }
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
    // Prefer everything in shared memory; drop the adjacency tables, then the
    // per-slot state, to global memory when the CTA would not fit.
    bool st_smem = state, tables_smem = true;
    SmemLayout L = smem_layout(C->n, C->m, P->t_max, C->dv_max, C->dc_max, adapt, st_smem, tables_smem);
    if (L.total > smem_optin) {
        tables_smem = false;
        L = smem_layout(C->n, C->m, P->t_max, C->dv_max, C->dc_max, adapt, st_smem, tables_smem);
    }
    if (L.total > smem_optin && st_smem) {
        st_smem = false;
        tables_smem = true;
        L = smem_layout(C->n, C->m, P->t_max, C->dv_max, C->dc_max, adapt, st_smem, tables_smem);
        if (L.total > smem_optin) {
            tables_smem = false;
            L = smem_layout(C->n, C->m, P->t_max, C->dv_max, C->dc_max, adapt, st_smem, tables_smem);
        }
    }
    if (L.total > smem_optin)
        return fail(NGDBF_ERR_UNSUPPORTED, "code too large for the shared-memory decision words");
    KernelFn fn = pick_kernel(P->variant, st_smem, C->dv_max > 7);
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, L.total);
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute");
    // Most resident warps per SM; ties go to more CTAs (more slots in flight).
    int best_block = 0, best_bps = 0, best_warps = -1;
    for (int block : {1024, 512, 256}) {
        int bps = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, fn, block, L.total);
        if (e != cudaSuccess) return cuda_fail(e, "cudaOccupancyMaxActiveBlocksPerMultiprocessor");
        const int warps = bps * block / 32;
        if (bps > 0 && (warps > best_warps || (warps == best_warps && bps > best_bps))) {
            best_block = block;
            best_bps = bps;
            best_warps = warps;
        }
    }
    if (best_bps == 0) return fail(NGDBF_ERR_UNSUPPORTED, "decode kernel does not fit on an SM");
    const int64_t groups = (n_frames + kSlots - 1) / kSlots;
    plan->block = best_block;
    plan->blocks_per_sm = best_bps;
    plan->grid = (int)std::min<int64_t>((int64_t)sm_count * best_bps, groups);
    plan->smem = L.total;
    plan->st_smem = st_smem;
    plan->tables_smem = tables_smem;
    *fn_out = fn;
    *sm_count_out = sm_count;
    (void)smem_per_sm;
    return NGDBF_OK;
}

// Kernel arguments of one decode: scratch at `base` (work counter, then the
// per-slot samples), per-slot state at `st_base` when it lives in global memory.
void fill_args(const ngdbf_code* C, const ngdbf_params* P, const LaunchPlan& plan, const float* y,
               int64_t n_frames, float sigma, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
               int32_t* iters, uint8_t* pass, unsigned char* base, unsigned char* st_base,
               bool st_global, DecodeArgs* out) {
    DecodeArgs& A = *out;
    std::memset(&A, 0, sizeof(A));
    A.n = C->n; A.m = C->m; A.dv_max = C->dv_max; A.dc_max = C->dc_max;
    A.chk_cols = C->d_chk_cols; A.sym_chks = C->d_sym_chks; A.sym_deg = C->d_sym_deg;
    A.tables_smem = plan.tables_smem ? 1 : 0;
    A.y = y; A.n_frames = n_frames; A.frame_offset = frame_offset;
    A.bits = bits; A.iters = iters; A.pass = pass; A.nb = (C->n + 7) / 8;
    A.w = P->w; A.theta = P->theta;
    A.scale = (float)((double)P->eta * (double)sigma);
    A.clamp = (P->y_max > 0.0f && std::isfinite(P->y_max)) ? 1 : 0;
    A.y_max = A.clamp ? P->y_max : 0.0f;
    A.t_max = P->t_max;
    A.t_smooth = std::max(0, P->t_max - P->smooth_window);
    A.queue = reinterpret_cast<unsigned long long*>(base);
    A.yslots = reinterpret_cast<float*>(base + 256);
    A.st_global = st_global ? reinterpret_cast<uint16_t*>(st_base) : nullptr;
    host_gen_consts(seed, A.G);
    double p = 1.0;
    for (int u = 0; u <= P->t_max; ++u) {
        A.thr[u] = (float)((double)P->theta * p);
        p = p * (double)P->lambda;
    }
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
    if (P->variant & ~3) return fail(NGDBF_ERR_INVALID_ARG, "unknown variant bits");
    if (P->precision != NGDBF_FP32) return fail(NGDBF_ERR_UNSUPPORTED, "only NGDBF_FP32 is implemented");
    if (P->q_bits != 0) return fail(NGDBF_ERR_INVALID_ARG, "q_bits is reserved and must be 0");
    return NGDBF_OK;
}

ngdbf_status decode_impl(const ngdbf_code* C, const float* y, int64_t n_frames, float sigma,
                         const ngdbf_params* P, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
                         int32_t* iters, uint8_t* pass, cudaStream_t stream) {
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
    const size_t slot_elems = (size_t)plan.grid * C->n * kSlots;
    const size_t bytes_y = (slot_elems * 4 + 255) / 256 * 256;
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

    e = cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), stream);
    if (e == cudaSuccess) {
        fn<<<plan.grid, plan.block, plan.smem, stream>>>(A);
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
    g_last_launch.grid = plan.grid;
    g_last_launch.block = plan.block;
    g_last_launch.smem_bytes = plan.smem;
    g_last_launch.state_in_smem = plan.st_smem ? 1 : 0;
    g_last_launch.kernels = 1;
    g_last_launch.sm_count = sm_count;
    return NGDBF_OK;
}

}  // namespace

extern "C" {

const char* ngdbf_last_error(void) { return g_last_error.c_str(); }

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
    if (chunk_frames <= 0) {
        // about 256 MB of samples per chunk, at least 4096 frames
        chunk_frames = std::max<int64_t>(4096, (int64_t)(256ll << 20) / (4 * n));
    }
    chunk_frames = std::min(chunk_frames, n_frames);
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
    for (int b = 0; b < 2 && rs == NGDBF_OK; ++b) {
        e = cudaStreamCreateWithFlags(&st[b], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&buf[b], per, pool, st[b]);
        if (e != cudaSuccess) rs = cuda_fail(e, "host decode set-up");
    }
    int64_t kernels = 0;
    for (int64_t off = 0, c = 0; off < n_frames && rs == NGDBF_OK; off += chunk_frames, ++c) {
        const int b = (int)(c & 1);
        const int64_t F = std::min(chunk_frames, n_frames - off);
        unsigned char* p = static_cast<unsigned char*>(buf[b]);
        float* dy = reinterpret_cast<float*>(p);
        uint8_t* dbits = p + align256(by);
        int32_t* diters = reinterpret_cast<int32_t*>(dbits + align256(bb));
        uint8_t* dpass = reinterpret_cast<uint8_t*>(diters) + align256(bi);
        e = cudaMemcpyAsync(dy, y_host + off * n, (size_t)F * n * 4, cudaMemcpyHostToDevice, st[b]);
        if (e != cudaSuccess) { rs = cuda_fail(e, "host-to-device copy"); break; }
        rs = decode_impl(C, dy, F, sigma, P, seed, frame_offset + (uint64_t)off, dbits, diters, dpass, st[b]);
        if (rs != NGDBF_OK) break;
        kernels += g_last_launch.kernels;
        e = cudaMemcpyAsync(bits_host + off * nb, dbits, (size_t)F * nb, cudaMemcpyDeviceToHost, st[b]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(iters_host + off, diters, (size_t)F * 4, cudaMemcpyDeviceToHost, st[b]);
        if (e == cudaSuccess) e = cudaMemcpyAsync(pass_host + off, dpass, (size_t)F, cudaMemcpyDeviceToHost, st[b]);
        if (e != cudaSuccess) rs = cuda_fail(e, "device-to-host copy");
    }
    for (int b = 0; b < 2; ++b) {
        if (buf[b]) cudaFreeAsync(buf[b], st[b]);
        if (st[b]) {
            cudaError_t es = cudaStreamSynchronize(st[b]);
            if (es != cudaSuccess && rs == NGDBF_OK) rs = cuda_fail(es, "stream synchronize");
            cudaStreamDestroy(st[b]);
        }
    }
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
    const size_t per_cta_y = (size_t)C->n * kSlots * 4;
    const size_t per_cta_st = (state && !plan.st_smem) ? (size_t)C->n * kSlots * 2 : 0;
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
    e = cudaMemsetAsync(A.queue, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_fail(e, "clearing the static work counter");
    fn<<<grid, plan.block, plan.smem, stream>>>(A);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "decode launch");
    g_last_launch.grid = grid;
    g_last_launch.block = plan.block;
    g_last_launch.smem_bytes = plan.smem;
    g_last_launch.state_in_smem = plan.st_smem ? 1 : 0;
    g_last_launch.kernels = 1;
    g_last_launch.sm_count = sm_count;
    return NGDBF_OK;
}
