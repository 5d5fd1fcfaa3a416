// ngdbf_kernels.cuh -- shared device code of the NGDBF decoder (sm_103a): job and launch
// descriptors, the shared-memory layout and the persistent slot loop for one job.
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
//      from a global atomic queue for them and loads those frames,
//   A'. adds, per symbol, the unsatisfied-check words of M(k) lane-wise (one
//      4-bit lane per slot; bit-sliced for symbol degrees above 7) into the
//      count of unsatisfied checks, shared by the 32 slots, then
//   C. runs Step 2 / Step 3b (or Step 3a) for every symbol of every live slot:
//      a warp processes four symbols (one Philox call) at a time with lane =
//      slot, reads the lane's count, forms E_k = x_k y_k + w S_k + q_k, compares
//      it with theta lambda^{u_k}, adapts u_k, accumulates the smoothing counter,
//      and rebuilds the decision word with a warp ballot.
// Slots therefore iterate independently (each frame has its own t), a
// converged frame frees its slot at once, and the CTA only stops when the
// queue is empty and its last slot finished.
//
// Per-(symbol, slot) state: the held sample (global scratch, L2-resident), and a
// 16-bit word holding u_k (bits 0-8) and the number of -1 decisions inside the
// smoothing window (bits 9-15), in shared memory when it fits, else in global
// scratch.  Both are laid out by groups of four symbols, [k/4][slot][k%4], so
// that phase C reads one vector per lane for the four symbols of a Philox call;
// the count words likewise ([k/4][slot quarter][k%4]) and the decision words
// are contiguous.  Decision and syndrome words, counts, the threshold and
// generator tables live in shared memory, the adjacency tables there when they fit.
#pragma once

#include <cooperative_groups.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <type_traits>

#include "../../include/ngdbf.h"
#include "ngdbf_device.cuh"

namespace ngdbf {

constexpr int kSlots = 32;

// Symbols rounded up to whole groups of four (the per-slot arrays are laid out by groups).
__host__ __device__ inline int pad4(int n) { return (n + 3) & ~3; }
// Index of (symbol k, slot f) in the group layout [k/4][slot][k%4].
__host__ __device__ inline int gidx(int k, int f) { return (((k >> 2) * kSlots + f) << 2) | (k & 3); }
constexpr int kTabChk = 1;              // N(i) table in shared memory
constexpr int kTabSym = 2;              // M(k) table and degrees in shared memory

constexpr int kMaxT = NGDBF_MAX_T;
constexpr uint32_t kUMask = 0x1FFu;   // u_k: bits 0-8
constexpr int kCShift = 9;            // smoothing count: bits 9-15

// Arithmetic of the held samples and of E_k (Sec. IV-E): the perturbation is
// always the FP32 generator output.
enum Precision { kFP32 = 0, kFP16 = 1, kFIX = 2, kFIXACC = 3 };
constexpr int kAccBits = 8;           // FIXACC: accumulator steps per half level = 2^8

template <int PREC> struct Held;
template <> struct Held<kFP32> { using T = float; };
template <> struct Held<kFP16> { using T = __half; };
template <> struct Held<kFIX> { using T = int8_t; };      // signed level code b, value 2b + 1
template <> struct Held<kFIXACC> { using T = int8_t; };   // the same Eq. 8 level code

// One decode job: a code, a batch of frames and the parameters of the method.
struct Job {
    // code tables (device)
    int32_t n, m, dv_max, dc_max;
    const uint16_t* chk_cols;   // [dc_max][m]   N(i) column-major, padded with n
    const uint16_t* sym_chks;   // [n][dv_max]   M(k) row-major, padded with m
    const uint8_t* sym_deg;     // [n]           d_v(k)
    // batch
    const float* y;             // [n_frames][n]
    int64_t n_frames;
    uint64_t frame_offset;
    uint8_t* bits;              // [n_frames][nb]
    int32_t* iters;
    uint8_t* pass;
    int32_t nb;
    // parameters
    float w, scale, y_max;      // w: FP32 value, or its binary16 value for FP16
    int32_t clamp, t_max, t_smooth;   // t_smooth = max(0, T - W)
    float fix_R;                // fixed point: fl32(2^Q / (2 Y_max)), kmax = 2^(Q-1) - 1, W~
    int32_t fix_kmax, fix_W;
    float acc_R;                // FIXACC: accumulator steps per unit fl32(2^(Q+8) / Y_max), w in steps
    int32_t acc_W;
    // thresholds theta lambda^u, u = 0..T: FP32 bits, binary16 values as FP32 bits, or
    // fixed-point levels Theta~(u) (FIX) or steps (FIXACC) as int32 (device memory; the
    // single-job launch passes them inline instead)
    const uint32_t* thr;
    unsigned long long* queue;  // next unclaimed frame of this job
    long long work;             // job tables: estimated work of one frame, n x (T + 1)
    int32_t single;             // Step 3a: flip only the symbol with the least E_k (ties: lowest k)
    int32_t uniform;            // Sec. V-B: uniform perturbation of the same variance
    // objective trace of frames 0 .. trace_frames-1 (nullptr: off): unsatisfied checks U(t) and
    // the correlation C(t) = sum_k rint(x_k y~_k 2^32), [frame][t_max + 1]
    int32_t* trace_u;
    long long* trace_c;
    long long trace_frames;
    double trace_yunit;         // FIX / FIXACC: value of one half level, Y_max 2^-Q
    // serving (0 / nullptr otherwise): `queue` holds (gen << 32) | frames claimed and claims
    // check the generation, so a CTA still holding an earlier job of the same ring slot never
    // takes frames of a later one; the CTA that finishes the last frame counts it in `done` and
    // writes `gen` into the host-visible word `notify`
    uint32_t gen;
    unsigned int* done;
    unsigned int* notify;
    const unsigned int* retire;     // serving: nonzero once the resident kernel is retiring (no claims)
    // serving: jobs with the same nonzero chain_key have the same code and decoding parameters
    // (they differ only in samples, sigma, frame offset, outputs and counters), so a CTA may
    // decode frames of several of them in its slots at once
    unsigned long long chain_key;
};

// Chaining of serving jobs inside one CTA (decode_job with CHAIN): the jobs whose frames the
// slots hold (entries of jl, slot f holds a frame of jl[slot_e[f]]), the entry frames are
// claimed from, and `next`, which finds another published job with the same chain_key.
constexpr int kChain = 8;
struct NoNext {
    __device__ bool operator()(unsigned long long, Job&) const { return false; }
};
template <class Next>
struct ChainCtx {
    Job* jl;                    // [kChain] shared memory
    int8_t* slot_e;             // [kSlots] shared memory
    int* cur_e;                 // shared memory
    Next next;
};

// Claims up to k consecutive frames of job A: returns true and the first frame id in *base
// (ids at or beyond A.n_frames mean no frame), or false when none is left.  Serving jobs
// (A.gen != 0) claim by compare-and-swap within their generation, at most kClaimTries times.
constexpr int kClaimTries = 4096;
__device__ __forceinline__ bool claim_frames(const Job& A, unsigned k, unsigned long long* base) {
    if (A.gen == 0u) {
        *base = atomicAdd(A.queue, (unsigned long long)k);
        return true;
    }
    // a retiring resident kernel takes no new frames: they wait for the next launch, which
    // has every CTA, instead of being decoded by the few CTAs still finishing
    if (A.retire != nullptr && *(const volatile unsigned int*)A.retire != 0u) return false;
    unsigned long long old = *(volatile unsigned long long*)A.queue;
    for (int it = 0; it < kClaimTries; ++it) {
        if ((uint32_t)(old >> 32) != A.gen || (long long)(uint32_t)old >= A.n_frames) return false;
        const unsigned long long got = atomicCAS(A.queue, old, old + k);
        if (got == old) {
            *base = (uint32_t)old;
            return true;
        }
        old = got;
    }
    return false;
}

// Launch of one job: the job and its thresholds travel as kernel parameters.
struct DecodeArgs {
    Job J;
    int32_t placement;          // adjacency tables copied into shared memory: kTabChk | kTabSym
    void* yslots;               // [grid][pad4(n)/4][32][4] held samples (4, 2 or 1 bytes each)
    uint16_t* st_global;        // [grid][pad4(n)/4][32][4] when the state is not in shared memory
    GenConsts G;
    uint32_t thr[kMaxT + 1];
};

// Launch of a job table: CTA c starts with job first_job[c] and, once that job has
// no unclaimed frame left and its slots are idle, moves to the job with the most
// unclaimed work (frames x Job::work).  Each job gets its own shared-memory layout
// (job_layout); the launch has room for the largest.
struct MultiArgs {
    const Job* jobs;
    int32_t n_jobs;
    const int32_t* first_job;   // [grid]
    int32_t n_max, m_max, t_max, dv_max, dc_max;   // layout maxima over the jobs
    int32_t placement;          // adjacency tables copied into shared memory: kTabChk | kTabSym
    // cluster launches: jobs with n >= split_min_n are split over the `cluster` CTAs of a
    // cluster (n_local symbols per CTA at most); the per-CTA arrays hold n_local symbols
    int32_t cluster, split_min_n, n_local;
    int32_t smem_bytes;         // dynamic shared memory of the launch (every job's layout fits)
    void* yslots;               // [grid][pad4(n_local)/4][32][4]
    uint16_t* st_global;        // [grid][pad4(n_local)/4][32][4] when the state is not in shared memory
    GenConsts G;
};

// Symbols one CTA decodes when the `size` CTAs of a cluster share one 32-slot group: [k_lo, k_hi),
// k_lo a multiple of 32 (size 1: the whole code).  Rank r of C takes chunks of 32 symbols
// [r nc / C, (r + 1) nc / C) of the nc = ceil(n / 32) chunks.
struct Split {
    int rank, size, k_lo, k_hi;
};
__host__ __device__ inline Split split_range(int rank, int size, int n) {
    const int nc = (n + 31) / 32;
    Split S;
    S.rank = rank;
    S.size = size;
    S.k_lo = 32 * (rank * nc / size);
    S.k_hi = 32 * ((rank + 1) * nc / size);
    if (S.k_hi > n) S.k_hi = n;
    return S;
}
// Largest number of symbols a CTA holds when a code of n symbols is split over `size` CTAs.
__host__ __device__ inline int split_local_max(int n, int size) { return 32 * (((n + 31) / 32 + size - 1) / size); }

struct SmemLayout {
    int32_t off_frame, off_start, off_ctl, off_best, off_trace, off_icdf, off_xw, off_sw, off_cnt, off_thr, off_st,
        off_chk, off_sym, total;
};

// Offsets in bytes of the shared-memory arrays.  ctl holds: [0..1] unsatisfied
// masks (double-buffered by pass parity), [2] live mask, [3] new-slot mask.
// When d_v <= 7 (narrow), sw holds per check four words with one 4-bit lane per slot
// (lane f & 7 of word f >> 3: 1 when check i is unsatisfied for slot f), and cnt holds
// per symbol, in the same lanes, S_k + 8 = d_v(k) + 8 - 2 (unsatisfied checks in M(k)),
// as words [k/4][quarter f >> 3][k%4] (16 bytes per symbol).  Otherwise (wide) sw holds
// the 32-bit unsatisfied mask of each check and cnt, per symbol, the bit-sliced count
// (seven words, bit f for slot f) and d_v(k) (32 bytes).  xw has room for whole groups
// and the zero sentinel word at index n.
// `wide` (< 0: from dv_max) selects the count and syndrome formats, which follow the kernel's
// WIDE template argument when a job table lays out a job of lower degree.
__host__ __device__ inline SmemLayout smem_layout(int n, int m, int t_max, int dv_max, int dc_max,
                                                  bool need_thr, bool st_smem, int tables, int n_local = -1,
                                                  int wide = -1) {
    if (n_local < 0) n_local = n;   // symbols whose counts, state and M(k) rows this CTA holds
    const bool wd = wide < 0 ? dv_max > 7 : wide != 0;
    SmemLayout L;
    int o = 0;
    auto take = [&](int bytes, int align) {
        o = (o + align - 1) / align * align;
        int r = o;
        o += bytes;
        return r;
    };
    const int cnt_bytes = wd ? 32 : 16;
    L.off_frame = take(kSlots * 8, 16);
    L.off_start = take(kSlots * 4, 16);
    L.off_ctl = take(8 * 4, 16);
    L.off_best = take(2 * kSlots * 8, 16); // single-bit variant: least (E key, k) per slot, two rounds
    L.off_trace = take(kSlots * 12, 16);   // objective trace: per slot C (int64), then U (int32)
    L.off_icdf = take(256 * 16, 16);       // inverse normal CDF coefficients
    L.off_cnt = take(pad4(n_local) * cnt_bytes, 16);
    L.off_xw = take(pad4(n + 1) * 4, 16);
    L.off_sw = take((m + 1) * (wd ? 4 : 16), 16);
    // all 512 values of the 9-bit u field: an idle slot's counter may pass T (its lookups are
    // don't-care but stay inside the table)
    L.off_thr = need_thr ? take((kUMask + 1) * 4, 16) : -1;
    L.off_st = st_smem ? take(pad4(n_local) * kSlots * 2, 16) : -1;
    L.off_chk = (tables & kTabChk) ? take(dc_max * m * 2, 16) : -1;
    L.off_sym = (tables & kTabSym) ? take(n_local * dv_max * 2 + n_local, 16) : -1;
    L.total = (o + 15) / 16 * 16;
    return L;
}

// Layout of one job of a job table: arrays sized for the job's own code (n_local symbols per
// CTA: its share when split over a cluster) in the launch's count and syndrome format, with
// as many of the adjacency tables that `tables` allows as fit in `bytes` (both, then N(i)
// alone, then none); *tables_out receives the placement taken.  Host planning and the kernel
// evaluate it alike, so the launch's shared memory is the largest job's, not the layout of
// the table's maxima.
__host__ __device__ inline SmemLayout job_layout(int n, int m, int t_max, int dv_max, int dc_max, bool need_thr,
                                                 bool st_smem, bool wide, int tables, int n_local, int bytes,
                                                 int* tables_out) {
    const int opts[3] = {tables & (kTabChk | kTabSym), tables & kTabChk, 0};
    SmemLayout L{};
    for (int i = 0; i < 3; ++i) {
        L = smem_layout(n, m, t_max, dv_max, dc_max, need_thr, st_smem, opts[i], n_local, wide ? 1 : 0);
        *tables_out = opts[i];
        if (L.total <= bytes) break;
    }
    return L;
}

// Signed fixed-point level code of v (Eq. 8): k = min(floor(|v| R), kmax) decided in FP32,
// b = k for v >= 0 and -k - 1 otherwise; the level's value is 2b + 1 in units of Delta/2.
__host__ __device__ inline int32_t fix_code(float v, float R, int32_t kmax) {
#ifdef __CUDA_ARCH__
    const float a = __fmul_rn(fabsf(v), R);
    const int32_t k = (a < (float)kmax) ? __float2int_rd(a) : kmax;
#else
    const float a = std::fabs(v) * R;
    const int32_t k = (a < (float)kmax) ? (int32_t)std::floor(a) : kmax;
#endif
    return v >= 0.0f ? k : -k - 1;
}

// Order-preserving 32-bit key of an FP32 value (-0 counts as +0, as a comparison would).
__device__ __forceinline__ uint32_t order_key(float v) {
    uint32_t b = __float_as_uint(v);
    if (b == 0x80000000u) b = 0u;
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// Bits 0..7 of b moved to bits 0, 4, ..., 28 (one bit per 4-bit lane).
__device__ __forceinline__ uint32_t spread_nibbles(uint32_t b) {
    b = (b | (b << 12)) & 0x000F000Fu;
    b = (b | (b << 6)) & 0x03030303u;
    return (b | (b << 3)) & 0x11111111u;
}

// Position of the (j+1)-th set bit of mask (j < popc(mask)).
__device__ __forceinline__ int nth_set_bit(uint32_t mask, int j) {
    for (int i = 0; i < j; ++i) mask &= mask - 1u;
    return __ffs(mask) - 1;
}

// Objective trace (Sec. III-B objective f(x) = sum_k x_k y_k + sum_i s_i): for the live slots whose
// frame id is below A.trace_frames, records at this syndrome test t the number of unsatisfied
// checks U(t) and C(t) = sum_k rint(x_k(t) y~_k 2^32) (each term exact in double; integer sums are
// independent of their order).  CTA-wide; every thread calls it with the same `live`.
template <int PREC>
__device__ __forceinline__ void trace_round(const Job& A, const SmemLayout& L, const uint16_t* chk_cols,
                                         const typename Held<PREC>::T* ys, uint32_t live, int round) {
    extern __shared__ __align__(16) unsigned char smem[];
    const long long* lane_frame = reinterpret_cast<const long long*>(smem + L.off_frame);
    const int32_t* lane_start = reinterpret_cast<const int32_t*>(smem + L.off_start);
    const uint32_t* xw = reinterpret_cast<const uint32_t*>(smem + L.off_xw);
    unsigned long long* tr_c = reinterpret_cast<unsigned long long*>(smem + L.off_trace);
    int32_t* tr_u = reinterpret_cast<int32_t*>(smem + L.off_trace + kSlots * 8);
    const int tid = threadIdx.x, lane = tid & 31;
    const bool mine = ((live >> lane) & 1u) && lane_frame[lane] >= 0 && lane_frame[lane] < A.trace_frames;
    const uint32_t tmask = __ballot_sync(0xFFFFFFFFu, mine);   // the same in every warp
    if (tmask == 0u) return;
    if (tid < kSlots) {
        tr_c[tid] = 0ull;
        tr_u[tid] = 0;
    }
    __syncthreads();
    const int n = A.n, m = A.m;
    // U(t): the syndrome words recomputed from the decision words
    for (int base = 0; base < m; base += blockDim.x) {
        const int i = base + tid;
        uint32_t s = 0u;
        if (i < m)
            for (int j = 0; j < A.dc_max; ++j) s ^= xw[chk_cols[j * m + i]];
        for (uint32_t r = tmask; r; r &= r - 1u) {
            const int f = __ffs(r) - 1;
            const int c = __popc(__ballot_sync(0xFFFFFFFFu, (s >> f) & 1u));
            if (lane == 0 && c) atomicAdd(tr_u + f, c);
        }
    }
    // C(t): sum over symbols of the signed held sample, scaled by 2^32 and rounded
    for (int base = 0; base < n; base += blockDim.x) {
        const int k = base + tid;
        for (uint32_t r = tmask; r; r &= r - 1u) {
            const int f = __ffs(r) - 1;
            long long term = 0;
            if (k < n) {
                double v;
                if constexpr (PREC == kFP32) {
                    v = (double)ys[gidx(k, f)];
                } else if constexpr (PREC == kFP16) {
                    v = (double)__half2float(ys[gidx(k, f)]);
                } else {
                    v = (double)(2 * (int32_t)ys[gidx(k, f)] + 1) * A.trace_yunit;
                }
                if ((xw[k] >> f) & 1u) v = -v;
                term = __double2ll_rn(v * 4294967296.0);
            }
#pragma unroll
            for (int o = 16; o; o >>= 1) term += __shfl_xor_sync(0xFFFFFFFFu, term, o);
            if (lane == 0 && term) atomicAdd(tr_c + f, (unsigned long long)term);
        }
    }
    __syncthreads();
    if (tid < kSlots && ((tmask >> tid) & 1u)) {
        const long long fr = lane_frame[tid];
        const size_t at = (size_t)fr * (size_t)(A.t_max + 1) + (size_t)(round - lane_start[tid]);
        A.trace_u[at] = tr_u[tid];
        A.trace_c[at] = (long long)tr_c[tid];
    }
    __syncthreads();
}

// The four held samples of one slot in a group (16, 8 or 4 bytes, aligned).
__device__ __forceinline__ void load_held4(const float* p, float v[4]) {
    const float4 a = *reinterpret_cast<const float4*>(p);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void load_held4(const __half* p, __half v[4]) {
    const uint2 a = *reinterpret_cast<const uint2*>(p);
    v[0] = __ushort_as_half((unsigned short)(a.x & 0xFFFFu));
    v[1] = __ushort_as_half((unsigned short)(a.x >> 16));
    v[2] = __ushort_as_half((unsigned short)(a.y & 0xFFFFu));
    v[3] = __ushort_as_half((unsigned short)(a.y >> 16));
}
__device__ __forceinline__ void load_held4(const int8_t* p, int8_t v[4]) {
    const uint32_t a = *reinterpret_cast<const uint32_t*>(p);
    v[0] = (int8_t)(a & 0xFFu); v[1] = (int8_t)((a >> 8) & 0xFFu);
    v[2] = (int8_t)((a >> 16) & 0xFFu); v[3] = (int8_t)(a >> 24);
}

// The slot loop for one job (rows a0-a8 of the method): CTA-wide, returns when the job
// has no unclaimed frame left and every slot of this CTA is idle.  `A` is the job (kernel
// parameters or a shared-memory copy), `thr_src` its thresholds, `L` the shared-memory
// layout of the launch, `ys`/`st_cta` this CTA's slot scratch.
//
// Thread 0 of a CTA whose slots chain serving jobs: gives the slots in `want` new frames,
// claimed from the current entry and, when its job has none left, from other published jobs
// with the same chain key, which ch.next copies into a free entry (one that no slot of `busy`
// or of those just filled refers to).  Sets lane_frame (frame index within its job; -1 for a
// slot left empty), lane_start = start and ch.slot_e for the filled slots; returns them.
template <class Next>
__device__ uint32_t fill_chained(ChainCtx<Next>& ch, unsigned long long key, uint32_t want, uint32_t busy,
                                 int start, long long* lane_frame, int32_t* lane_start) {
    uint32_t fresh = 0;
    for (int step = 0; step <= kChain; ++step) {
        const uint32_t left = want & ~fresh;
        if (!left) break;
        const Job& E = ch.jl[*ch.cur_e];
        const int k = __popc(left);
        unsigned long long base = 0;
        if (claim_frames(E, (unsigned)k, &base)) {
            for (int j = 0; j < k; ++j) {
                const int f = nth_set_bit(left, j);
                const unsigned long long fid = base + j;
                if (fid < (unsigned long long)E.n_frames) {
                    lane_frame[f] = (long long)fid;
                    lane_start[f] = start;
                    ch.slot_e[f] = (int8_t)*ch.cur_e;
                    fresh |= 1u << f;
                }
            }
        }
        if (!(want & ~fresh) || key == 0ull) break;
        // the current job has no frames left: another with the same key, into a free entry
        const uint32_t held = busy | fresh;
        int e2 = -1;
        for (int e = 0; e < kChain && e2 < 0; ++e) {
            if (e == *ch.cur_e) continue;
            bool used = false;
            for (uint32_t r = held; r; r &= r - 1) used |= ch.slot_e[__ffs(r) - 1] == e;
            if (!used) e2 = e;
        }
        if (e2 < 0 || !ch.next(key, ch.jl[e2])) break;
        *ch.cur_e = e2;
    }
    for (uint32_t r = want & ~fresh; r; r &= r - 1) lane_frame[__ffs(r) - 1] = -1;
    return fresh;
}

// Cluster split (CL, S.size > 1): the S.size CTAs of a thread-block cluster decode the same
// 32 slots, each the symbols [S.k_lo, S.k_hi) (samples, state, counts and M(k) rows of those
// only), with a full copy of the decision words in every CTA: each computes all syndromes (so
// the stop vote is the same everywhere), writes the decision words it changes into every
// copy through distributed shared memory, and rank 0 claims frames for the cluster and
// writes the slot table into every CTA.  Cluster barriers separate the phases; every CTA
// takes the same branches (they depend only on the vote and the slot table), so all of them
// reach every barrier.
//
// Chaining (CHAIN, serving): A is ch.jl[0]; when A has no unclaimed frame left, free slots take
// frames of other published jobs with A's chain key (fill_chained), so the CTA keeps its slots
// busy across requests instead of waiting for A's slowest frame; the loop returns when no such
// job has frames left and every slot is idle.
template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE, int PREC, bool CL = false, bool CHAIN = false,
          class Next = NoNext>
__device__ __forceinline__ void decode_job(const Job& A, const uint32_t* thr_src, const GenConsts& G,
                                           const SmemLayout& L, int tables,
                                           typename Held<PREC>::T* ys, uint16_t* st_cta,
                                           Split S = Split{0, 1, 0, 0},
                                           ChainCtx<Next> ch = ChainCtx<Next>{nullptr, nullptr, nullptr, Next{}}) {
    static_assert(!(CL && CHAIN), "chained jobs are not split over clusters");
    constexpr bool kState = ADAPT || SMOOTH;
    // the job whose frame slot f holds (per-request fields: samples, sigma, frame offset,
    // outputs, counters); every other field is the same for all chained jobs
    auto job_of = [&](int f) -> const Job& {
        if constexpr (CHAIN) return ch.jl[ch.slot_e[f]];
        return A;
    };
    using HeldT = typename Held<PREC>::T;
    extern __shared__ __align__(16) unsigned char smem[];
    const int n = A.n, m = A.m, T = A.t_max, dv_max = A.dv_max, dc_max = A.dc_max;
    const bool split = CL && S.size > 1;
    const int k_lo = split ? S.k_lo : 0, k_hi = split ? S.k_hi : n;   // this CTA's symbols
    const int nl = k_hi - k_lo;
    // barrier over the CTAs that share the slots (the cluster when split, else this CTA)
    auto group_sync = [&]() {
        if constexpr (CL) {
            if (split) {
                cooperative_groups::this_cluster().sync();
                return;
            }
        }
        __syncthreads();
    };
    // the same shared-memory word in another CTA of the cluster
    auto peer = [&](auto* p, int r) { return cooperative_groups::this_cluster().map_shared_rank(p, r); };
    long long* lane_frame = reinterpret_cast<long long*>(smem + L.off_frame);
    int32_t* lane_start = reinterpret_cast<int32_t*>(smem + L.off_start);
    uint32_t* ctl = reinterpret_cast<uint32_t*>(smem + L.off_ctl);
    uint4* cnt = reinterpret_cast<uint4*>(smem + L.off_cnt);
    uint32_t* xw = reinterpret_cast<uint32_t*>(smem + L.off_xw);
    uint32_t* sw = reinterpret_cast<uint32_t*>(smem + L.off_sw);
    unsigned long long* best = reinterpret_cast<unsigned long long*>(smem + L.off_best);
    float4* icdf = reinterpret_cast<float4*>(smem + L.off_icdf);
    uint32_t* thr = ADAPT ? reinterpret_cast<uint32_t*>(smem + L.off_thr) : nullptr;
    uint16_t* st = nullptr;
    if constexpr (kState) {
        st = ST_SMEM ? reinterpret_cast<uint16_t*>(smem + L.off_st) : st_cta;
    }
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    // adjacency tables: only phases A and A' read them, so a generic pointer to
    // shared or global memory serves both placements
    const uint16_t* chk_cols = A.chk_cols;
    const uint16_t* sym_chks = A.sym_chks;
    const uint8_t* sym_deg = A.sym_deg;
    if (tables & kTabChk) {
        uint16_t* c = reinterpret_cast<uint16_t*>(smem + L.off_chk);
        for (int i = tid; i < dc_max * m; i += blockDim.x) c[i] = A.chk_cols[i];
        chk_cols = c;
    }
    int sym_base = 0;           // first symbol of the M(k) rows sym_chks points to
    if (tables & kTabSym) {
        uint16_t* s = reinterpret_cast<uint16_t*>(smem + L.off_sym);
        uint8_t* d = reinterpret_cast<uint8_t*>(s + nl * dv_max);
        for (int i = tid; i < nl * dv_max; i += blockDim.x) s[i] = A.sym_chks[k_lo * dv_max + i];
        for (int i = tid; i < nl; i += blockDim.x) d[i] = A.sym_deg[k_lo + i];
        sym_chks = s;
        sym_deg = d;
        sym_base = k_lo;
    }

    // ---- the first 32 frames, then the set-up: generator table, zeroed state, sentinels,
    // thresholds.  Unsplit, the claim comes first, so that a CTA that finds every frame taken
    // (several CTAs pick a job at once) returns without the set-up. ----
    auto claim_first = [&]() {          // thread 0 (rank 0 when split): slot table and live mask
        uint32_t live = 0;
        for (int c = 0; c < 8; ++c) ctl[c] = 0u;
        if constexpr (CHAIN) {
            *ch.cur_e = 0;
            for (int f = 0; f < kSlots; ++f) ch.slot_e[f] = 0;     // every slot names a loaded entry
            live = fill_chained(ch, A.chain_key, 0xFFFFFFFFu, 0u, 0, lane_frame, lane_start);
        } else {
            unsigned long long base = 0;
            const bool got = claim_frames(A, kSlots, &base);
            for (int f = 0; f < kSlots; ++f) {
                const unsigned long long fid = base + f;
                lane_start[f] = 0;
                if (got && fid < (unsigned long long)A.n_frames) {
                    lane_frame[f] = (long long)fid;
                    live |= 1u << f;
                } else {
                    lane_frame[f] = -1;
                }
            }
        }
        ctl[2] = live;
        ctl[3] = live;
        return live;
    };
    if (!split) {
        if (tid == 0) claim_first();
        __syncthreads();
        if (ctl[2] == 0u) return;
    }
    for (int i = tid; i < 256; i += blockDim.x) icdf[i] = G.icdf[i];
    for (int k = tid; k < pad4(n + 1); k += blockDim.x) xw[k] = 0u;
    for (int i = tid; i < (m + 1) * (WIDE ? 1 : 4); i += blockDim.x) sw[i] = 0u;
    // a serving job's thresholds and samples were copied in while the kernel runs: read them
    // past L1, which may still hold lines of an earlier request at the same addresses
    if constexpr (ADAPT)
        for (int u = tid; u <= T; u += blockDim.x) thr[u] = A.gen ? __ldcg(thr_src + u) : thr_src[u];
    // threshold of the non-adaptive variants; chained jobs read it once here, since the first
    // job's memory is returned when that job completes
    const uint32_t th0_once = CHAIN ? __ldcg(thr_src) : 0u;
    if constexpr (kState)
        for (int e = tid; e < pad4(nl) * kSlots; e += blockDim.x) st[e] = 0;
    if (tid < 2 * kSlots) best[tid] = ~0ull;
    if (split) {
        group_sync();        // every copy cleared before rank 0 writes the slot table
        if (tid == 0 && S.rank == 0) {
            const uint32_t live = claim_first();
            if constexpr (CL) {
                for (int r = 0; r < S.size; ++r) {
                    if (r == S.rank) continue;
                    long long* pf = peer(lane_frame, r);
                    int32_t* ps = peer(lane_start, r);
                    uint32_t* pc = peer(ctl, r);
                    for (int f = 0; f < kSlots; ++f) {
                        pf[f] = lane_frame[f];
                        ps[f] = 0;
                    }
                    for (int c = 0; c < 8; ++c) pc[c] = 0u;
                    pc[2] = live;
                    pc[3] = live;
                }
            }
        }
    }
    group_sync();

    int round = 0;   // flip phases executed by this CTA; slot f is at t = round - lane_start[f]
    int pass_id = 0;
    bool refill = true;
    for (;;) {
        if (refill) {
            // ---- load new frames: saturated samples into the slot columns, x(0) = sign(y) ----
            const uint32_t fresh = ctl[3];
            for (int k = k_lo + tid; k < k_hi; k += blockDim.x) {
                uint32_t word = xw[k] & ~fresh;
                uint32_t rest = fresh;
                while (rest) {
                    const int f = __ffs(rest) - 1;
                    rest &= rest - 1;
                    const Job& Jf = job_of(f);
                    const float* yp = Jf.y + (size_t)lane_frame[f] * n + k;
                    float v = Jf.gen ? __ldcg(yp) : __ldg(yp);
                    if (A.clamp) {
                        if (v > A.y_max) v = A.y_max;
                        if (v < -A.y_max) v = -A.y_max;
                    }
                    bool negative;
                    const int at = gidx(k - k_lo, f);
                    if constexpr (PREC == kFP32) {
                        ys[at] = v;
                        negative = !(v >= 0.0f);
                    } else if constexpr (PREC == kFP16) {
                        const __half h = __float2half_rn(v);
                        ys[at] = h;
                        negative = !(__half2float(h) >= 0.0f);        // sign(-0) = +1
                    } else {
                        const int32_t b = fix_code(v, A.fix_R, A.fix_kmax);
                        ys[at] = (int8_t)b;
                        negative = b < 0;
                    }
                    if (negative) word |= 1u << f;
                    if constexpr (kState) st[at] = 0;
                }
                xw[k] = word;
                if constexpr (CL) {
                    for (int r = 0; split && r < S.size; ++r)
                        if (r != S.rank) peer(xw, r)[k] = word;
                }
            }
            group_sync();
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
                if constexpr (WIDE) {
                    if (i < m && sub == 0) sw[i] = s;
                } else {
                    // byte `sub` of the word, one slot per 4-bit lane (slots 8 sub .. 8 sub + 7)
                    if (i < m) sw[4 * i + sub] = spread_nibbles((s >> (8 * sub)) & 0xFFu);
                }
                acc |= s;
            }
            acc = __reduce_or_sync(0xFFFFFFFFu, acc);
            if (lane == 0 && acc) atomicOr(unsat, acc);
            __syncthreads();
        }
        const uint32_t unsat = ctl[pass_id & 1];
        ++pass_id;
        uint32_t live = ctl[2];
        if (A.trace_u != nullptr)
            trace_round<PREC>(A, L, chk_cols, ys, live, round);
        const uint32_t conv = live & ~unsat;
        const int my_t = round - lane_start[lane];
        const uint32_t at_T = __ballot_sync(0xFFFFFFFFu, ((live >> lane) & 1u) && my_t >= T);
        const uint32_t fin = conv | (live & at_T);

        if (fin) {
            // ---- B. outputs of finished slots ----
            const int nfin = __popc(fin);
            const int b_lo = k_lo >> 3, nbl = ((k_hi + 7) >> 3) - b_lo;   // this CTA's output bytes
            const int work = nfin * nbl;
            for (int idx = tid; idx < work; idx += blockDim.x) {
                const int j = idx / nbl, b = b_lo + (idx - j * nbl);
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
                                const int neg = (int)(st[gidx(k - k_lo, f)] >> kCShift) + (int)bit;
                                const int X = terms - 2 * neg;
                                bit = X < 0 ? 1u : (X > 0 ? 0u : bit);
                            }
                        }
                        byte |= bit << q;
                    }
                }
                job_of(f).bits[(size_t)lane_frame[f] * A.nb + b] = (uint8_t)byte;
            }
            if (tid < nfin && (!split || S.rank == 0)) {
                const int f = nth_set_bit(fin, tid);
                const bool ok = (conv >> f) & 1u;
                const long long fr = lane_frame[f];
                const Job& Jf = job_of(f);
                Jf.iters[fr] = ok ? round - lane_start[f] : T;
                Jf.pass[fr] = ok ? 1 : 0;
            }
            if (A.done != nullptr) __threadfence();   // outputs visible before they are counted
            group_sync();           // every CTA is done with the finished slots' table entries
            if (A.done != nullptr && tid == 0 && (!split || S.rank == 0)) {
                if constexpr (CHAIN) {
                    // the finished frames counted in their own jobs
                    for (int e = 0; e < kChain; ++e) {
                        int cnt = 0;
                        for (uint32_t r = fin; r; r &= r - 1)
                            cnt += ch.slot_e[__ffs(r) - 1] == e ? 1 : 0;
                        if (!cnt) continue;
                        const Job& E = ch.jl[e];
                        const unsigned int before = atomicAdd(E.done, (unsigned int)cnt);
                        if ((long long)before + cnt == E.n_frames) {
                            __threadfence_system();
                            *(volatile unsigned int*)E.notify = E.gen;
                        }
                    }
                } else {
                    const unsigned int before = atomicAdd(A.done, (unsigned int)nfin);
                    if ((long long)before + nfin == A.n_frames) {
                        __threadfence_system();
                        *(volatile unsigned int*)A.notify = A.gen;
                    }
                }
            }
            // ---- claim new frames for the finished slots ----
            if (tid == 0 && (!split || S.rank == 0)) {
                uint32_t fresh = 0;
                if constexpr (CHAIN) {
                    fresh = fill_chained(ch, A.chain_key, fin, live & ~fin, round, lane_frame, lane_start);
                } else {
                    unsigned long long base = 0;
                    const bool got = claim_frames(A, (unsigned)nfin, &base);
                    for (int j = 0; j < nfin; ++j) {
                        const int f = nth_set_bit(fin, j);
                        const unsigned long long fid = base + j;
                        if (got && fid < (unsigned long long)A.n_frames) {
                            lane_frame[f] = (long long)fid;
                            lane_start[f] = round;
                            fresh |= 1u << f;
                        } else {
                            lane_frame[f] = -1;
                        }
                    }
                }
                ctl[2] = (live & ~fin) | fresh;
                ctl[3] = fresh;
                if constexpr (CL) {
                    for (int r = 0; split && r < S.size; ++r) {
                        if (r == S.rank) continue;
                        long long* pf = peer(lane_frame, r);
                        int32_t* ps = peer(lane_start, r);
                        uint32_t* pc = peer(ctl, r);
                        for (int j = 0; j < nfin; ++j) {
                            const int f = nth_set_bit(fin, j);
                            pf[f] = lane_frame[f];
                            ps[f] = lane_start[f];
                        }
                        pc[2] = ctl[2];
                        pc[3] = ctl[3];
                    }
                }
            }
            group_sync();
            live = ctl[2];
            if (ctl[3]) {
                refill = true;      // new frames need their t = 0 syndrome test first
                continue;
            }
        }
        if (live == 0) break;

        // ---- A'. per symbol and slot, the count of unsatisfied checks in M(k) ----
        for (int k = k_lo + tid; k < k_hi; k += blockDim.x) {
            const int kk = k - k_lo;                      // local index of the symbol
            const uint16_t* row = sym_chks + (k - sym_base) * dv_max;
            if constexpr (!WIDE) {
                // d_v <= 7: one 4-bit lane per slot, counts added lane-wise without carries;
                // stored as S_k + 8 = d_v + 8 - 2 count in [1, 15]
                const uint4* sw4 = reinterpret_cast<const uint4*>(sw);
                uint4 c = make_uint4(0u, 0u, 0u, 0u);
                for (int e = 0; e < dv_max; ++e) {
                    const uint4 s = sw4[row[e]];
                    c.x += s.x; c.y += s.y; c.z += s.z; c.w += s.w;
                }
                const uint32_t D = ((uint32_t)sym_deg[k - sym_base] + 8u) * 0x11111111u;
                uint32_t* cw = reinterpret_cast<uint32_t*>(cnt) + ((kk >> 2) << 4) + (kk & 3);
                cw[0] = D - 2u * c.x;     // quarter q of the group at word 4 q + k % 4
                cw[4] = D - 2u * c.y;
                cw[8] = D - 2u * c.z;
                cw[12] = D - 2u * c.w;
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
                cnt[2 * kk] = make_uint4(b[0], b[1], b[2], b[3]);
                cnt[2 * kk + 1] = make_uint4(b[4], b[5], b[6], (uint32_t)sym_deg[k - sym_base]);
            }
        }
        __syncthreads();

        // ---- C. Step 2 and Step 3b for every symbol of every live slot ----
        {
            const bool act = (live >> lane) & 1u;
            const long long fr = lane_frame[lane];
            const Job& Jl = job_of(lane);           // an idle lane's entry is stale: don't-care
            const uint64_t fid = Jl.frame_offset + (uint64_t)(act ? fr : 0);
            const uint32_t flo = (uint32_t)fid, fhi = (uint32_t)(fid >> 32);
            const int t = act ? round - lane_start[lane] : 0;
            const bool window = SMOOTH && act && t >= A.t_smooth;
            const int g_lo = k_lo >> 2;              // first group of this CTA's symbols
            // threshold of the non-adaptive variants
            const uint32_t th0 = CHAIN ? th0_once : (A.gen ? __ldcg(thr_src) : thr_src[0]);
            const float scale = Jl.scale, wgt = A.w, fix_R = A.fix_R, acc_R = A.acc_R;
            const int32_t fix_kmax = A.fix_kmax, fix_W = A.fix_W, acc_W = A.acc_W;
            const bool uniform = A.uniform != 0;
            const bool single = !ADAPT && A.single;
            const uint32_t nib_shift = 4u * (lane & 7);
            const float wgt_m8 = -8.0f * wgt;       // exact
            unsigned long long my_best = ~0ull;      // single-bit variant: (E key << 32) | k
            // one group of four symbols; only the last group of a code with n % 4 != 0 is partial
            // (its missing symbols read the zeroed padding and are skipped)
            auto group = [&](const int gl, auto partial_tag) {
                constexpr bool kPartial = decltype(partial_tag)::value;
                const int g = g_lo + gl;                  // group index in the code (Philox counter)
                const int k0 = 4 * g;
                const int at = (gl * kSlots + lane) * 4;  // this lane's entries in the group layout
                // issue the sample, state, count, decision-word and threshold loads (one vector
                // each) before the generator's arithmetic, so that their latency overlaps it
                HeldT yv[4];
                load_held4(ys + at, yv);
                [[maybe_unused]] uint32_t sv[4], cwv[4], thv[4];
                if constexpr (kState) {
                    const uint2 s2 = *reinterpret_cast<const uint2*>(st + at);
                    sv[0] = s2.x & 0xFFFFu; sv[1] = s2.x >> 16; sv[2] = s2.y & 0xFFFFu; sv[3] = s2.y >> 16;
                }
                if constexpr (!WIDE) {
                    const uint4 c4 = reinterpret_cast<const uint4*>(cnt)[gl * 4 + (lane >> 3)];
                    cwv[0] = c4.x; cwv[1] = c4.y; cwv[2] = c4.z; cwv[3] = c4.w;
                }
                const uint4 x4 = reinterpret_cast<const uint4*>(xw)[g];
                const uint32_t xwv[4] = {x4.x, x4.y, x4.z, x4.w};
                if constexpr (ADAPT) {
                    // u_k <= t - 1 < T for a live slot (cleared on every refill)
#pragma unroll
                    for (int j = 0; j < 4; ++j) thv[j] = thr[sv[j] & kUMask];
                }
                float z[4];
                noise4((uint32_t)g, (uint32_t)t, flo, fhi, G, icdf, uniform, z);
                uint32_t fmv[4] = {0u, 0u, 0u, 0u};          // flip masks of the four symbols
                [[maybe_unused]] uint32_t nvv[4];             // new state words
                if constexpr (kState) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) nvv[j] = sv[j];
                }
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int k = k0 + j;
                    if (kPartial && k >= n) break;
                    int S;
                    float ws;           // fl(w S_k)
                    if constexpr (!WIDE) {
                        // this slot's 4-bit lane of the symbol's count word: S_k + 8, and
                        // w S_k = fl(w (S_k + 8) - 8 w) in one rounding (8 w is exact)
                        const uint32_t nib = (cwv[j] >> nib_shift) & 0xFu;
                        S = (int)nib - 8;
                        ws = __fmaf_rn(wgt, __uint2float_rn(nib), wgt_m8);
                    } else {
                        const uint4 c = cnt[2 * (k - k_lo)], d = cnt[2 * (k - k_lo) + 1];
                        const int unsat_cnt = (int)(((c.x >> lane) & 1u) | (((c.y >> lane) & 1u) << 1) |
                                                    (((c.z >> lane) & 1u) << 2) | (((c.w >> lane) & 1u) << 3) |
                                                    (((d.x >> lane) & 1u) << 4) | (((d.y >> lane) & 1u) << 5) |
                                                    (((d.z >> lane) & 1u) << 6));
                        S = (int)d.w - 2 * unsat_cnt;
                        ws = __fmul_rn(wgt, __int2float_rn(S));
                    }
                    const uint32_t xword = xwv[j];
                    // x_k = -1 as the sign bit of x_k y_k, and as a bool
                    const uint32_t xsign = (xword << (31 - lane)) & 0x80000000u;
                    [[maybe_unused]] const bool xneg = xsign != 0u;
                    const float q = __fmul_rn(scale, z[j]);
                    // E_k = ((x_k y_k) + w S_k) + q_k, rounded after every operation (Step 2)
                    auto metric32 = [&]() -> float {
                        const float xy = __uint_as_float(__float_as_uint((float)yv[j]) ^ xsign);
                        return __fadd_rn(__fadd_rn(xy, ws), q);
                    };
                    // the same in binary16: each result rounded to binary16.  fl(w S_k) is the
                    // exact product of a binary16 w and a small integer; the additions are
                    // binary16 additions (a correctly rounded FP32 addition of binary16
                    // operands rounded once more to binary16 gives the same value)
                    [[maybe_unused]] auto metric16 = [&]() -> __half {
                        if constexpr (PREC == kFP16) {
                            const __half xy = __ushort_as_half(__half_as_ushort(yv[j]) ^ (uint16_t)(xsign >> 16));
                            return __hadd(__hadd(xy, __float2half_rn(ws)), __float2half_rn(q));
                        } else {
                            return __float2half_rn(0.0f);
                        }
                    };
                    // the held Eq. 8 level in accumulator steps (2^8 per half level), plus the
                    // weight and the perturbation rounded to steps: exact int32
                    [[maybe_unused]] auto metric_acc = [&]() -> int32_t {
                        const int32_t Y = (2 * (int32_t)yv[j] + 1) * (1 << kAccBits);
                        const int32_t Qs = __float2int_rn(__fmul_rn(q, acc_R));
                        return (xneg ? -Y : Y) + acc_W * S + Qs;
                    };
                    // below_threshold(u): E_k < theta_k in the held arithmetic
                    auto below = [&](uint32_t th_bits) -> bool {
                        if constexpr (PREC == kFP32) {
                            return metric32() < __uint_as_float(th_bits);
                        } else if constexpr (PREC == kFP16) {
                            return __half2float(metric16()) < __uint_as_float(th_bits);
                        } else if constexpr (PREC == kFIX) {
                            // Eq. 9 in units of Delta/2, exact integers
                            const int32_t Y = 2 * (int32_t)yv[j] + 1;
                            const int32_t Qv = 2 * fix_code(q, fix_R, fix_kmax) + 1;
                            return (xneg ? -Y : Y) + fix_W * S + Qv < (int32_t)th_bits;
                        } else {
                            return metric_acc() < (int32_t)th_bits;
                        }
                    };
                    if constexpr (!ADAPT) {
                        if (single) {
                            // Step 3a: remember this lane's least E_k; flips wait for all symbols
                            uint32_t key;
                            if constexpr (PREC == kFP32) {
                                key = order_key(metric32());
                            } else if constexpr (PREC == kFP16) {
                                key = order_key(__half2float(metric16()));
                            } else if constexpr (PREC == kFIXACC) {
                                key = (uint32_t)metric_acc() ^ 0x80000000u;
                            } else {
                                const int32_t Y = 2 * (int32_t)yv[j] + 1;
                                const int32_t Qv = 2 * fix_code(q, fix_R, fix_kmax) + 1;
                                key = (uint32_t)((xneg ? -Y : Y) + fix_W * S + Qv) ^ 0x80000000u;
                            }
                            const unsigned long long cand = ((unsigned long long)key << 32) | (uint32_t)k;
                            my_best = cand < my_best ? cand : my_best;
                            if constexpr (SMOOTH) {
                                if (window && xneg) nvv[j] = sv[j] + (1u << kCShift);
                            }
                            continue;
                        }
                    }
                    bool flip;
                    if constexpr (kState) {
                        const uint32_t s0 = sv[j];
                        const uint32_t th = ADAPT ? thv[j] : th0;
                        const bool lower = below(th);       // evaluated for every lane, no branch
                        // an idle slot (no frame) may flip and count too: its decision bits and
                        // counters are cleared when it takes a frame and never reach an output
                        flip = lower;
                        // u_k += 1 when not flipped; the window counter counts x_k = -1
                        nvv[j] = s0 + ((ADAPT && !flip) ? 1u : 0u) + (window ? (xsign >> (31 - kCShift)) : 0u);
                    } else {
                        flip = below(th0);              // idle slots: don't-care, as above
                    }
                    fmv[j] = __ballot_sync(0xFFFFFFFFu, flip);
                }
                if constexpr (kState) {
                    const uint2 n2 = make_uint2(nvv[0] | (nvv[1] << 16), nvv[2] | (nvv[3] << 16));
                    if (ADAPT || nvv[0] != sv[0] || nvv[1] != sv[1] || nvv[2] != sv[2] || nvv[3] != sv[3])
                        *reinterpret_cast<uint2*>(st + at) = n2;
                }
                // Step 3b flips of the group (the single-bit variant flips after the sweep)
                if (lane == 0 && !single) {
                    const uint4 nw = make_uint4(xwv[0] ^ fmv[0], xwv[1] ^ fmv[1], xwv[2] ^ fmv[2], xwv[3] ^ fmv[3]);
                    reinterpret_cast<uint4*>(xw)[g] = nw;
                    if constexpr (CL) {
                        for (int r = 0; split && r < S.size; ++r)
                            if (r != S.rank) reinterpret_cast<uint4*>(peer(xw, r))[g] = nw;
                    }
                }
            };
            const int full = nl >> 2, groups_l = (nl + 3) >> 2;   // only the code's last group can be partial
            for (int gl = warp; gl < full; gl += nwarps) group(gl, std::false_type{});
            if (full < groups_l && warp == full % nwarps) group(full, std::true_type{});
            if constexpr (!ADAPT) {
                // the least (E key, k) of each slot over this CTA's symbols; when split, in the
                // buffer of this round's parity (the CTAs of the cluster read each other's)
                unsigned long long* bcur = best + (split ? (round & 1) * kSlots : 0);
                if (single && act) atomicMin(bcur + lane, my_best);
            }
        }
        if constexpr (!ADAPT) {
            if (!ADAPT && A.single) {
                group_sync();
                // each live slot flips its least-E_k symbol (the lowest k among equal values), in
                // every copy of the decision words
                unsigned long long* bcur = best + (split ? (round & 1) * kSlots : 0);
                if (tid < kSlots) {
                    unsigned long long b = bcur[tid];
                    if constexpr (CL) {
                        for (int r = 0; split && r < S.size; ++r) {
                            if (r == S.rank) continue;
                            const unsigned long long o = *peer(bcur + tid, r);
                            b = o < b ? o : b;
                        }
                    }
                    if ((live >> tid) & 1u) atomicXor(xw + (uint32_t)b, 1u << tid);
                    // clear the buffer of the next round (when split, the other CTAs finished
                    // reading it before the previous round's closing barrier)
                    best[(split ? ((round + 1) & 1) * kSlots : 0) + tid] = ~0ull;
                }
            }
        }
        group_sync();
        ++round;
    }
}

}  // namespace ngdbf
