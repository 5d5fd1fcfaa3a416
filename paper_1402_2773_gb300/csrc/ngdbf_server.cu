// ngdbf_server.cu -- the serving loop: continuous batching of decode requests on a resident
// persistent kernel.
//
// Requests (a code, host samples and host outputs) are queued in arrival order.  A scheduler
// thread admits them while the device memory they need fits the budget: it takes a block from
// the library's stream-ordered pool, copies the samples (staged, like ngdbf_decode_host, unless
// direct copies are selected) and thresholds in on one of the copy streams, and publishes the
// request into a ring of job descriptors in device memory (small ordered copies from a
// page-locked mirror, made to wait for the request's own copies).  One persistent job-table
// kernel serves the ring: whenever a CTA has no
// frames left in its current request it takes the oldest published request with unclaimed
// frames, so requests that arrive while others are on the GPU join the running launch as
// CTAs -- and, inside a request, slots -- free up.  The CTA that finishes a request's last frame
// writes the request's generation into a completion word in page-locked host memory; the
// scheduler then copies the outputs back and returns the request's memory to the budget.  Idle
// CTAs poll the ring (in device memory, backing off); the first that has found no work for
// about 20 ms retires the whole kernel (every CTA leaves, none takes new frames), and the
// scheduler launches the kernel again when new work is published.  A request whose code needs
// a larger shared-memory layout, or another variant or precision, than the running kernel
// waits until it drains.  While the kernel runs only copy-engine operations are issued (the one
// memset clears the retire word between launches), so nothing waits behind it for SMs.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "ngdbf_host.h"

namespace ngdbf {

constexpr int kRing = 1024;                       // descriptor slots: requests on the device at once, at most
constexpr long long kIdleNs = 20'000'000;         // a CTA this long without work retires the kernel

// In device memory; written only by copies from the host's page-locked mirror.
struct ServeRing {
    unsigned long long tail;          // requests [0, tail) are published
    unsigned long long head;          // requests below head are complete (where scans start)
    unsigned int stop_epoch;          // the kernel of epoch e exits at once when stop_epoch >= e,
    unsigned int drain_epoch;         // and when it has no work left when drain_epoch >= e
    unsigned long long ready[kRing];  // q + 1 while the slot holds the complete descriptor of request q
    Job jobs[kRing];
};

// Page-locked staging of one ring slot (free again once the slot's request completes).
struct SlotStage {
    unsigned long long claim0;        // (gen << 32) | 0
    unsigned int done0;               // 0
    unsigned int pad;
    unsigned long long ready0, ready1, tail1;   // 0, seq + 1, seq + 1
    Job desc;
    uint32_t thr[NGDBF_MAX_T + 1];
};

struct ServeArgs {
    const ServeRing* ring;            // device memory
    unsigned int* notify;             // [kRing] page-locked, mapped: a slot's generation once done
    // device, zeroed before each launch: set by the first CTA that has been idle long enough;
    // then every CTA leaves at its next pick and no CTA claims new frames, so the kernel exits
    // as a whole (CTAs leaving one by one would leave it running on a few of them)
    unsigned int* retire;
    unsigned int epoch;
    int32_t n_max, m_max, t_max, dv_max, dc_max, placement;
    int32_t smem_bytes;               // the launch's dynamic shared memory
    void* yslots;                     // [grid][pad4(n_max)/4][32][4]
    uint16_t* st_global;              // [grid][pad4(n_max)/4][32][4] when the state is not in shared memory
    GenConsts G;
};

// A CTA chains to another request only while at least kChainMinPending published requests have
// unclaimed frames (the server is saturated: chaining keeps slots busy across requests), and
// only to one among the kChainWindow oldest of those, so that requests of other codes are not
// overtaken without bound; with fewer pending, the picker takes requests in arrival order.
constexpr int kChainMinPending = 16;
constexpr int kChainWindow = 32;

// Finds, for a CTA whose request has no frames left, another published request with the same
// chain key and unclaimed frames (the oldest) and copies its descriptor into `out` (thread 0).
// A search that failed is not repeated for the same key until more requests are published.
struct RingNext {
    const volatile ServeRing* R;
    unsigned long long* fail;           // shared memory: [0] the ring tail, [1] the key of the last failed search
    __device__ bool operator()(unsigned long long key, Job& out) const {
        const unsigned long long tail = R->tail, head = R->head;
        if (tail == fail[0] && key == fail[1]) return false;
        int pending = 0, found = -1;
        uint32_t found_gen = 0;
        unsigned long long found_q = 0;
        for (unsigned long long q = head; q < tail && q < head + kRing; ++q) {
            const int slot = (int)(q % kRing);
            if (R->ready[slot] != q + 1) continue;
            __threadfence();
            const uint32_t gen = R->jobs[slot].gen;
            const long long frames = R->jobs[slot].n_frames;
            unsigned long long* queue = R->jobs[slot].queue;
            const unsigned long long c = *(volatile unsigned long long*)queue;
            if ((uint32_t)(c >> 32) != gen || (long long)(uint32_t)c >= frames) continue;
            if (++pending > kChainWindow) break;
            if (found < 0 && R->jobs[slot].chain_key == key) {
                found = slot;
                found_gen = gen;
                found_q = q;
            }
            if (found >= 0 && pending >= kChainMinPending) break;
        }
        if (found >= 0 && pending >= kChainMinPending) {     // (pending counts at most kChainWindow + 1)
            const volatile uint32_t* src = reinterpret_cast<const volatile uint32_t*>(&R->jobs[found]);
            uint32_t* dst = reinterpret_cast<uint32_t*>(&out);
            for (int w = 0; w < (int)(sizeof(Job) / 4); ++w) dst[w] = src[w];
            __threadfence();
            if (R->ready[found] == found_q + 1 && out.gen == found_gen) return true;
        }
        fail[0] = tail;
        fail[1] = key;
        return false;
    }
};

// The resident serving kernel: each CTA repeatedly takes the oldest published request that
// still has unclaimed frames (of its own generation) and runs the slot loop on it, chaining
// further requests of the same code and parameters into its free slots.  Every request is
// decoded in a shared-memory layout of its own code within the launch's bytes: with ST_SMEM
// (the largest code's state fits) the state is always in shared memory; otherwise a request
// whose code's state fits keeps it there too (in the 4-bit count format), and only the others
// use the global slot state.
template <bool ADAPT, bool SMOOTH, bool ST_SMEM, bool WIDE, int PREC>
__global__ void __launch_bounds__(1024) ngdbf_serve_kernel(const __grid_constant__ ServeArgs A) {
    using HeldT = typename Held<PREC>::T;
    constexpr bool kState = ADAPT || SMOOTH;
    __shared__ Job jl[kChain];      // jl[0]: the request picked; the others: chained requests
    __shared__ int8_t slot_e[kSlots];
    __shared__ int cur_e;
    __shared__ unsigned long long fail[2];
    Job& job = jl[0];
    if (threadIdx.x == 0) fail[0] = fail[1] = ~0ull;
    __shared__ int pick;
    HeldT* ys = static_cast<HeldT*>(A.yslots) + (size_t)blockIdx.x * pad4(A.n_max) * kSlots;
    uint16_t* st = A.st_global ? A.st_global + (size_t)blockIdx.x * pad4(A.n_max) * kSlots : nullptr;
    const volatile ServeRing* R = A.ring;
    long long slept = 0;
    unsigned int nap = 500;
    for (;;) {
        if (threadIdx.x == 0) {
            int p = -1;
            if (R->stop_epoch >= A.epoch || *(volatile unsigned int*)A.retire != 0u) {
                p = -2;
            } else {
                const unsigned long long tail = R->tail;
                const unsigned long long head = R->head;
                for (unsigned long long q = head; q < tail && q < head + kRing; ++q) {
                    const int slot = (int)(q % kRing);
                    // the slot must hold request q, complete, before and after the descriptor
                    // is read (the copies clear `ready` before they rewrite a slot)
                    if (R->ready[slot] != q + 1) continue;
                    __threadfence();
                    const uint32_t gen = R->jobs[slot].gen;
                    const long long frames = R->jobs[slot].n_frames;
                    unsigned long long* queue = R->jobs[slot].queue;
                    const unsigned long long c = *(volatile unsigned long long*)queue;
                    if ((uint32_t)(c >> 32) != gen || (long long)(uint32_t)c >= frames) continue;
                    // the descriptor word by word past L1 (the slot held earlier requests)
                    const volatile uint32_t* src = reinterpret_cast<const volatile uint32_t*>(&R->jobs[slot]);
                    uint32_t* dst = reinterpret_cast<uint32_t*>(&job);
                    for (int w = 0; w < (int)(sizeof(Job) / 4); ++w) dst[w] = src[w];
                    __threadfence();
                    if (R->ready[slot] != q + 1 || job.gen != gen) continue;
                    p = slot;
                    break;
                }
                if (p < 0 && R->drain_epoch >= A.epoch) p = -2;
                if (p < 0 && slept > kIdleNs) {                 // idle long enough: the kernel retires
                    atomicExch(A.retire, 1u);
                    p = -2;
                }
                if (p < 0) {
                    __nanosleep(nap);
                    slept += nap;
                    nap = nap < 64000u ? 2 * nap : nap;
                }
            }
            pick = p;
        }
        __syncthreads();
        const int p = pick;
        __syncthreads();
        if (p == -2) break;
        if (p < 0) continue;
        slept = 0;
        nap = 500;
        int tables = 0;
        const ChainCtx<RingNext> ch{jl, slot_e, &cur_e, RingNext{R, fail}};
        bool done = false;
        if constexpr (kState && !ST_SMEM && !WIDE) {
            const SmemLayout Ls = job_layout(job.n, job.m, job.t_max, job.dv_max, job.dc_max, ADAPT, true, WIDE,
                                             A.placement, job.n, A.smem_bytes, &tables);
            if (Ls.total <= A.smem_bytes) {
                decode_job<ADAPT, SMOOTH, true, WIDE, PREC, false, true, RingNext>(
                    job, job.thr, A.G, Ls, tables, ys, nullptr, Split{0, 1, 0, 0}, ch);
                done = true;
            }
        }
        if (!done) {
            // (a code no larger than the kind's maxima always fits without its state)
            const SmemLayout L = job_layout(job.n, job.m, job.t_max, job.dv_max, job.dc_max, ADAPT,
                                            ST_SMEM && kState, WIDE, A.placement, job.n, A.smem_bytes, &tables);
            decode_job<ADAPT, SMOOTH, ST_SMEM, WIDE, PREC, false, true, RingNext>(
                job, job.thr, A.G, L, tables, ys, st, Split{0, 1, 0, 0}, ch);
        }
        __syncthreads();
    }
}

namespace {

using ServeFn = void (*)(ServeArgs);

template <bool AD, bool SM, int PREC>
ServeFn serve_width(bool st_smem, bool wide) {
    if (st_smem) return wide ? ngdbf_serve_kernel<AD, SM, true, true, PREC> : ngdbf_serve_kernel<AD, SM, true, false, PREC>;
    return wide ? ngdbf_serve_kernel<AD, SM, false, true, PREC> : ngdbf_serve_kernel<AD, SM, false, false, PREC>;
}

template <int PREC>
ServeFn serve_variant(int variant, bool st_smem, bool wide) {
    switch (variant & 3) {
        case 0: return serve_width<false, false, PREC>(st_smem, wide);
        case 1: return serve_width<true, false, PREC>(st_smem, wide);
        case 2: return serve_width<false, true, PREC>(st_smem, wide);
        default: return serve_width<true, true, PREC>(st_smem, wide);
    }
}

ServeFn serve_kernel_fn(int variant, int precision, bool st_smem, bool wide) {
    switch (precision) {
        case NGDBF_FP16: return serve_variant<kFP16>(variant, st_smem, wide);
        case NGDBF_FIX: return serve_variant<kFIX>(variant, st_smem, wide);
        case NGDBF_FIXACC: return serve_variant<kFIXACC>(variant, st_smem, wide);
        default: return serve_variant<kFP32>(variant, st_smem, wide);
    }
}

}  // namespace
}  // namespace ngdbf

using namespace ngdbf;
using namespace ngdbf::host;

namespace {

double now_s() {
    using clk = std::chrono::steady_clock;
    static const clk::time_point t0 = clk::now();
    return std::chrono::duration<double>(clk::now() - t0).count();
}

struct Request {
    uint64_t id = 0;
    ngdbf_job job{};                 // y, bits, iters and pass are HOST pointers here
    const float* y_host = nullptr;
    uint8_t* bits_host = nullptr;
    int32_t* iters_host = nullptr;
    uint8_t* pass_host = nullptr;
    double t_submit = 0, t_done = 0;
    int32_t status = NGDBF_OK;
    // on the device
    uint64_t seq = 0;                // position in the ring
    int slot = -1;
    uint32_t gen = 0;
    int stream = 0;
    unsigned char* block = nullptr;  // samples | outputs | thresholds
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;        // copies in done, then copies out done
    Job dj{};                        // the descriptor the kernel reads
};

// Kind of the resident kernel: the template it instantiates and its shared-memory maxima.
struct Kind {
    int variant = -1, precision = -1;   // variant & 3 (ADAPT, SMOOTH) and the precision
    int n = 0, m = 0, t_max = 0, dv = 0, dc = 0;
    bool fits(const ngdbf_job& q) const {
        return (q.params.variant & 3) == variant && q.params.precision == precision && q.code->n <= n &&
               q.code->m <= m && q.params.t_max <= t_max && q.code->dv_max <= dv && q.code->dc_max <= dc &&
               ((q.code->dv_max > 7) == (dv > 7));
    }
};

}  // namespace

struct ngdbf_server {
    int device = 0;
    size_t budget = 0;
    int max_resident = 1;
    uint64_t seed = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;       // copy streams
    std::vector<Staging*> stages;            // per copy stream, staged copies of request samples
    std::map<std::string, unsigned long long> chain_ids;   // (code, params) -> chain key
    cudaStream_t pub_stream = nullptr;       // ring updates, in ring order
    cudaStream_t serve_stream = nullptr;     // the resident kernel
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> pending;            // arrival order
    std::vector<Request*> published;         // in the ring (copies in may still be running)
    std::vector<Request*> leaving;           // copies out in flight
    std::vector<Request*> completed;         // not yet reported by poll
    ServeRing* d_ring = nullptr;             // device memory
    unsigned int* notify_host = nullptr;     // [kRing] page-locked, mapped
    unsigned int* notify_dev = nullptr;
    SlotStage* stage = nullptr;              // [kRing] page-locked
    unsigned long long* head_img = nullptr;  // page-locked words copied into the ring
    unsigned int* epoch_img = nullptr;       // [2]: stop, drain
    unsigned long long* d_claim = nullptr;   // [kRing] (gen << 32) | frames claimed
    unsigned int* d_done = nullptr;          // [kRing] frames done
    unsigned int* d_retire = nullptr;        // set by the resident kernel when it retires
    uint32_t slot_gen[kRing] = {};
    uint64_t next_seq = 0, head = 0;
    std::vector<uint64_t> done_seq;          // completed sequence numbers above head
    // the resident kernel
    bool running = false;
    unsigned int epoch = 0;
    Kind kind;
    std::vector<Kind> seen;                  // per variant and precision: the largest layout so far
    size_t kind_scratch = 0;                 // scratch the kernel of `kind` takes at launch
    cudaEvent_t ev_kernel = nullptr;
    unsigned char* scratch = nullptr;
    size_t scratch_bytes = 0;
    int rr = 0;
    size_t in_use = 0;
    ngdbf_server_stats stats{};
    bool stop = false;
    std::thread worker;
};

namespace {

size_t request_bytes(const ngdbf_job& q) {
    const int64_t n = q.code->n, nb = (n + 7) / 8;
    return align256((size_t)q.n_frames * n * 4) + align256((size_t)q.n_frames * nb) +
           align256((size_t)q.n_frames * 4) + align256((size_t)q.n_frames) + align256((size_t)(q.params.t_max + 1) * 4);
}

void finish(ngdbf_server* S, Request* r, int32_t status) {
    r->t_done = now_s();
    r->status = status;
    S->completed.push_back(r);
    S->stats.completed += 1;
    if (status != NGDBF_OK) S->stats.failed += 1;
    else S->stats.frames += r->job.n_frames;
}

// Copies a request in and publishes it into the ring once its copies are done (every step is
// an asynchronous copy or an event wait: nothing here needs an SM).
ngdbf_status admit(ngdbf_server* S, Request* r) {
    const int si = S->rr++ % (int)S->streams.size();
    cudaStream_t st = S->streams[si];
    r->stream = si;
    r->bytes = request_bytes(r->job);
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&r->block), r->bytes, S->pool, st);
    if (e != cudaSuccess) { cudaGetLastError(); r->block = nullptr; return fail(NGDBF_ERR_OOM, "server: device block"); }
    const ngdbf_job& q = r->job;
    const int64_t n = q.code->n, nb = (n + 7) / 8, F = q.n_frames;
    unsigned char* p = r->block;
    float* dy = reinterpret_cast<float*>(p);
    p += align256((size_t)F * n * 4);
    uint8_t* dbits = p;
    p += align256((size_t)F * nb);
    int32_t* diters = reinterpret_cast<int32_t*>(p);
    p += align256((size_t)F * 4);
    uint8_t* dpass = p;
    p += align256((size_t)F);
    uint32_t* dthr = reinterpret_cast<uint32_t*>(p);
    r->seq = S->next_seq++;
    r->slot = (int)(r->seq % kRing);
    r->gen = ++S->slot_gen[r->slot];
    if (r->gen == 0) r->gen = ++S->slot_gen[r->slot];      // 0 marks a plain job
    SlotStage& sg = S->stage[r->slot];
    fill_job(q.code, &q.params, dy, F, q.sigma, q.frame_offset, dbits, diters, dpass, S->d_claim + r->slot, &r->dj,
             sg.thr);
    r->dj.thr = dthr;
    r->dj.gen = r->gen;
    // requests of the same code and parameters share a chain key: the kernel decodes frames
    // of several of them in one CTA's slots (they differ only in samples, sigma, offset, outputs)
    {
        std::string k(reinterpret_cast<const char*>(&q.code), sizeof(q.code));
        k.append(reinterpret_cast<const char*>(&q.params), sizeof(q.params));
        auto it = S->chain_ids.find(k);
        if (it == S->chain_ids.end()) it = S->chain_ids.emplace(k, (unsigned long long)S->chain_ids.size() + 1).first;
        r->dj.chain_key = it->second;
    }
    r->dj.done = S->d_done + r->slot;
    r->dj.retire = S->d_retire;
    r->dj.notify = S->notify_dev + r->slot;
    sg.claim0 = (unsigned long long)r->gen << 32;
    sg.done0 = 0;
    sg.ready0 = 0;
    sg.ready1 = r->seq + 1;
    sg.tail1 = r->seq + 1;
    sg.desc = r->dj;
    __atomic_store_n(&S->notify_host[r->slot], 0u, __ATOMIC_RELEASE);
    // the samples through the stream's staging buffers (host threads + copies from reused
    // page-locked memory) unless direct copies were asked for
    if (host_copy_mode() == NGDBF_HOST_COPY_STAGED && !S->stages[si]) S->stages[si] = staging_acquire(S->device);
    if (host_copy_mode() == NGDBF_HOST_COPY_STAGED && S->stages[si])
        e = staged_h2d(S->stages[si], dy, r->y_host, (size_t)F * n * 4, st);
    else
        e = cudaMemcpyAsync(dy, r->y_host, (size_t)F * n * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dthr, sg.thr, ((size_t)q.params.t_max + 1) * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_claim + r->slot, &sg.claim0, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(S->d_done + r->slot, &sg.done0, 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && !r->ev) e = cudaEventCreateWithFlags(&r->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
    // publication, in ring order, after the request's own copies: the slot invalid, the
    // descriptor, the slot valid for request seq, the tail
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->pub_stream, r->ev, 0);
    ServeRing* R = S->d_ring;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&R->ready[r->slot], &sg.ready0, 8, cudaMemcpyHostToDevice, S->pub_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&R->jobs[r->slot], &sg.desc, sizeof(Job), cudaMemcpyHostToDevice, S->pub_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&R->ready[r->slot], &sg.ready1, 8, cudaMemcpyHostToDevice, S->pub_stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&R->tail, &sg.tail1, 8, cudaMemcpyHostToDevice, S->pub_stream);
    if (e != cudaSuccess) return cuda_fail(e, "server: copy in");
    return NGDBF_OK;
}

// Launch plan of the resident kernel of a kind: shared-memory plan, grid and scratch bytes.
struct ServePlan {
    SmemPlan sp;
    int grid = 0;
    size_t per_y = 0, per_st = 0, bytes = 0;
};
ngdbf_status plan_serve(ngdbf_server* S, const Kind& K, ServePlan* out) {
    const bool state = (K.variant & 3) != 0, adapt = (K.variant & NGDBF_ADAPT) != 0, wide = K.dv > 7;
    ngdbf_status s = plan_smem(S->device, K.n, K.m, K.t_max, K.dv, K.dc, adapt, state,
                               (const void*)serve_kernel_fn(K.variant, K.precision, true, wide),
                               (const void*)serve_kernel_fn(K.variant, K.precision, false, wide), &out->sp);
    if (s != NGDBF_OK) return s;
    int sms = 0;
    cudaError_t e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, S->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    out->grid = sms * out->sp.bps;
    out->per_y = (size_t)pad4(K.n) * kSlots * held_bytes(K.precision);
    out->per_st = (state && !out->sp.st_smem) ? (size_t)pad4(K.n) * kSlots * 2 : 0;
    out->bytes = align256((size_t)out->grid * out->per_y) + align256((size_t)out->grid * out->per_st);
    return NGDBF_OK;
}

// Launches the resident kernel for the kind of the published requests (a new epoch).
ngdbf_status launch_kernel(ngdbf_server* S) {
    const Kind& K = S->kind;
    const bool wide = K.dv > 7;
    ServePlan P;
    ngdbf_status s = plan_serve(S, K, &P);
    if (s != NGDBF_OK) return s;
    const SmemPlan& sp = P.sp;
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&S->scratch), P.bytes, S->pool, S->serve_stream);
    if (e != cudaSuccess) { cudaGetLastError(); S->scratch = nullptr; return fail(NGDBF_ERR_OOM, "server: kernel scratch"); }
    S->scratch_bytes = P.bytes;
    ServeArgs A;
    std::memset(&A, 0, sizeof(A));
    A.ring = S->d_ring;
    A.notify = S->notify_dev;
    A.retire = S->d_retire;
    A.epoch = ++S->epoch;
    A.n_max = K.n; A.m_max = K.m; A.t_max = K.t_max; A.dv_max = K.dv; A.dc_max = K.dc;
    A.placement = sp.placement;
    A.smem_bytes = sp.smem;
    A.yslots = S->scratch;
    A.st_global = P.per_st ? reinterpret_cast<uint16_t*>(S->scratch + align256((size_t)P.grid * P.per_y)) : nullptr;
    host_gen_consts(S->seed, A.G);
    // the previous kernel retired (or drained): clear the word before this one starts; and the
    // kernel must see every ring update published so far
    e = cudaMemsetAsync(S->d_retire, 0, sizeof(unsigned int), S->pub_stream);
    if (e == cudaSuccess) e = cudaEventRecord(S->ev_kernel, S->pub_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(S->serve_stream, S->ev_kernel, 0);
    if (e == cudaSuccess) {
        serve_kernel_fn(K.variant, K.precision, sp.st_smem, wide)<<<P.grid, sp.block, sp.smem, S->serve_stream>>>(A);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(S->ev_kernel, S->serve_stream);
    if (e != cudaSuccess) {
        cudaFreeAsync(S->scratch, S->serve_stream);
        S->scratch = nullptr;
        return cuda_fail(e, "server: kernel launch");
    }
    S->running = true;
    S->in_use += P.bytes;
    S->stats.launches += 1;
    return NGDBF_OK;
}

// The kind a kernel needs for the first request to admit: the largest layout of its variant and
// precision seen so far (so that the kernel rarely has to drain for a larger code).
Kind kind_for(ngdbf_server* S, const Request* first) {
    const ngdbf_job& f = first->job;
    Kind* K = nullptr;
    for (Kind& k : S->seen)
        if (k.variant == (f.params.variant & 3) && k.precision == f.params.precision && (k.dv > 7) == (f.code->dv_max > 7))
            K = &k;
    if (!K) {
        S->seen.push_back(Kind());
        K = &S->seen.back();
        K->variant = f.params.variant & 3;
        K->precision = f.params.precision;
    }
    auto grow = [&](const ngdbf_job& q) {
        if ((q.params.variant & 3) != K->variant || q.params.precision != K->precision ||
            (q.code->dv_max > 7) != (K->dv > 7 || f.code->dv_max > 7))
            return;
        K->n = std::max(K->n, q.code->n);
        K->m = std::max(K->m, q.code->m);
        K->t_max = std::max(K->t_max, q.params.t_max);
        K->dv = std::max(K->dv, q.code->dv_max);
        K->dc = std::max(K->dc, q.code->dc_max);
    };
    grow(f);
    for (Request* r : S->pending) grow(r->job);
    return *K;
}

void copy_word(ngdbf_server* S, void* dst, const void* src, size_t bytes) {
    if (cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, S->pub_stream) != cudaSuccess) cudaGetLastError();
}

void scheduler(ngdbf_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        bool progressed = false;
        // 1. requests whose last frame is done: copy the outputs out
        for (size_t i = 0; i < S->published.size();) {
            Request* r = S->published[i];
            if (__atomic_load_n(&S->notify_host[r->slot], __ATOMIC_ACQUIRE) != r->gen) { ++i; continue; }
            cudaStream_t st = S->streams[r->stream];
            const int64_t F = r->job.n_frames, nb = (r->job.code->n + 7) / 8;
            cudaError_t e = cudaMemcpyAsync(r->bits_host, r->dj.bits, (size_t)F * nb, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->iters_host, r->dj.iters, (size_t)F * 4, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(r->pass_host, r->dj.pass, (size_t)F, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaEventRecord(r->ev, st);
            if (e != cudaSuccess) { cudaGetLastError(); r->status = NGDBF_ERR_CUDA; }
            S->leaving.push_back(r);
            S->published.erase(S->published.begin() + i);
            progressed = true;
        }
        // 2. outputs written: the request is complete, its memory and ring slot free
        for (size_t i = 0; i < S->leaving.size();) {
            Request* r = S->leaving[i];
            if (r->status == NGDBF_OK && cudaEventQuery(r->ev) == cudaErrorNotReady) { ++i; continue; }
            cudaGetLastError();
            cudaFreeAsync(r->block, S->streams[r->stream]);
            cudaEventDestroy(r->ev);
            r->ev = nullptr;
            S->in_use -= r->bytes;
            S->done_seq.push_back(r->seq);
            finish(S, r, r->status);
            S->leaving.erase(S->leaving.begin() + i);
            progressed = true;
        }
        // the scan start of the kernel: the oldest sequence number not yet complete
        std::sort(S->done_seq.begin(), S->done_seq.end());
        size_t adv = 0;
        while (adv < S->done_seq.size() && S->done_seq[adv] == S->head + adv) ++adv;
        if (adv) {
            S->head += adv;
            S->done_seq.erase(S->done_seq.begin(), S->done_seq.begin() + adv);
            *S->head_img = S->head;             // a copy may read a later head: still valid
            copy_word(S, &S->d_ring->head, S->head_img, 8);
        }
        // 3. the resident kernel exited (idle, drained or stopped)
        if (S->running && cudaEventQuery(S->ev_kernel) != cudaErrorNotReady) {
            cudaGetLastError();
            S->running = false;
            // freed on the publication stream, not on the kernel's: the pool lets later
            // allocations reuse a block by waiting for the freeing stream's work, and the
            // kernel's stream would by then run the next resident kernel, which only exits
            // when it runs out of work (requests' copies would wait for it)
            cudaFreeAsync(S->scratch, S->pub_stream);
            S->scratch = nullptr;
            S->in_use -= S->scratch_bytes;
            S->scratch_bytes = 0;
            progressed = true;
        }
        // 4. admission in arrival order, while memory, ring slots and the kernel's kind allow
        while (!S->pending.empty() && !S->stop) {
            Request* r = S->pending.front();
            if (r->job.n_frames == 0) {
                S->pending.pop_front();
                finish(S, r, NGDBF_OK);
                progressed = true;
                continue;
            }
            const size_t bytes = request_bytes(r->job);
            const bool on_device = S->running || !S->published.empty();
            if (on_device && !S->kind.fits(r->job)) {
                // another kind or a larger code: let the running work drain first
                if (S->running && S->epoch_img[1] != S->epoch) {
                    S->epoch_img[1] = S->epoch;
                    copy_word(S, &S->d_ring->drain_epoch, &S->epoch_img[1], 4);
                }
                break;
            }
            if (S->next_seq - S->head >= (uint64_t)S->max_resident) break;
            Kind K = S->kind;
            if (!on_device) {
                K = kind_for(S, r);
                ServePlan P;
                if (plan_serve(S, K, &P) != NGDBF_OK) {
                    S->pending.pop_front();
                    finish(S, r, NGDBF_ERR_UNSUPPORTED);
                    progressed = true;
                    continue;
                }
                S->kind_scratch = P.bytes;
            }
            const size_t reserve = S->running ? 0 : S->kind_scratch;   // scratch of a kernel still to be launched
            if (S->in_use + reserve + bytes > S->budget) {
                if (!on_device && reserve + bytes > S->budget) {          // can never run
                    S->pending.pop_front();
                    finish(S, r, NGDBF_ERR_OOM);
                    progressed = true;
                    continue;
                }
                break;                                   // wait for memory to be returned
            }
            if (!on_device) S->kind = K;
            S->pending.pop_front();
            ngdbf_status s = admit(S, r);
            if (s != NGDBF_OK) {
                // nothing of it was published: give its slot and memory back
                cudaStreamSynchronize(S->streams[r->stream]);
                if (r->block) cudaFreeAsync(r->block, S->streams[r->stream]);
                if (r->ev) { cudaEventDestroy(r->ev); r->ev = nullptr; }
                S->done_seq.push_back(r->seq);
                finish(S, r, s);
            } else {
                S->in_use += r->bytes;
                if (S->running) S->stats.admitted_into_running += 1;
                S->published.push_back(r);
                S->stats.peak_requests_on_device =
                    std::max<int32_t>(S->stats.peak_requests_on_device, (int32_t)S->published.size());
                S->stats.peak_bytes_in_use = std::max<int64_t>(
                    S->stats.peak_bytes_in_use, (int64_t)(S->in_use + (S->running ? 0 : S->kind_scratch)));
            }
            progressed = true;
        }
        // 5. published work and no kernel: launch one
        if (!S->running && !S->published.empty() && !S->stop) {
            ngdbf_status s = launch_kernel(S);
            if (s != NGDBF_OK) {
                // nothing can decode these: report them once their copies are done
                cudaStreamSynchronize(S->pub_stream);
                for (Request* r : S->published) {
                    cudaFreeAsync(r->block, S->streams[r->stream]);
                    if (r->ev) { cudaEventDestroy(r->ev); r->ev = nullptr; }
                    S->in_use -= r->bytes;
                    S->done_seq.push_back(r->seq);
                    finish(S, r, s);
                }
                S->published.clear();
            }
            S->stats.peak_bytes_in_use = std::max<int64_t>(S->stats.peak_bytes_in_use, (int64_t)S->in_use);
            progressed = true;
        }
        if (progressed) S->cv.notify_all();
        if (S->stop && S->published.empty() && S->leaving.empty() && !S->running) break;
        S->cv.wait_for(lk, std::chrono::microseconds(S->running ? 50 : 200));
    }
}

}  // namespace

extern "C" ngdbf_status ngdbf_server_create(size_t device_budget_bytes, int32_t max_inflight_launches,
                                            int32_t max_jobs_per_launch, uint64_t seed, ngdbf_server_t** out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (device_budget_bytes == 0) return fail(NGDBF_ERR_INVALID_ARG, "budget must be > 0");
    if (max_inflight_launches < 1 || max_inflight_launches > 16)
        return fail(NGDBF_ERR_INVALID_ARG, "max_inflight_launches (copy streams) must be 1..16");
    if (max_jobs_per_launch < 1 || max_jobs_per_launch > 4096)
        return fail(NGDBF_ERR_INVALID_ARG, "max_jobs_per_launch must be 1..4096");
    ngdbf_server* S = new (std::nothrow) ngdbf_server;
    if (!S) return fail(NGDBF_ERR_OOM, "host allocation");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) { delete S; return cuda_fail(e, "cudaGetDevice"); }
    ngdbf_status s = get_pool(S->device, &S->pool);
    if (s != NGDBF_OK) { delete S; return s; }
    S->budget = device_budget_bytes;
    S->max_resident = std::min(max_jobs_per_launch, kRing);
    S->seed = seed;
    e = cudaHostAlloc(reinterpret_cast<void**>(&S->notify_host), sizeof(unsigned int) * kRing, cudaHostAllocMapped);
    if (e == cudaSuccess) {
        std::memset(S->notify_host, 0, sizeof(unsigned int) * kRing);
        e = cudaHostGetDevicePointer(reinterpret_cast<void**>(&S->notify_dev), S->notify_host, 0);
    }
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&S->stage), sizeof(SlotStage) * kRing, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&S->head_img), 8, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void**>(&S->epoch_img), 8, cudaHostAllocDefault);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_ring, sizeof(ServeRing));
    if (e == cudaSuccess) e = cudaMalloc(&S->d_claim, sizeof(unsigned long long) * kRing);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_done, sizeof(unsigned int) * kRing);
    if (e == cudaSuccess) e = cudaMalloc(&S->d_retire, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(S->d_retire, 0, sizeof(unsigned int));
    if (e == cudaSuccess) e = cudaMemset(S->d_ring, 0, sizeof(ServeRing));
    if (e == cudaSuccess) e = cudaMemset(S->d_claim, 0, sizeof(unsigned long long) * kRing);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S->ev_kernel, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->serve_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&S->pub_stream, cudaStreamNonBlocking);
    for (int k = 0; k < max_inflight_launches && e == cudaSuccess; ++k) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e == cudaSuccess) S->streams.push_back(st);
        if (e == cudaSuccess) S->stages.push_back(nullptr);
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
        if (S->serve_stream) cudaStreamDestroy(S->serve_stream);
        if (S->pub_stream) cudaStreamDestroy(S->pub_stream);
        if (S->ev_kernel) cudaEventDestroy(S->ev_kernel);
        cudaFree(S->d_ring);
        cudaFree(S->d_claim);
        cudaFree(S->d_done);
        cudaFree(S->d_retire);
        if (S->stage) cudaFreeHost(S->stage);
        if (S->head_img) cudaFreeHost(S->head_img);
        if (S->epoch_img) cudaFreeHost(S->epoch_img);
        if (S->notify_host) cudaFreeHost(S->notify_host);
        delete S;
        return cuda_fail(e, "server set-up");
    }
    S->epoch_img[0] = S->epoch_img[1] = 0;
    S->worker = std::thread(scheduler, S);
    *out = S;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_server_submit(ngdbf_server_t* S, const ngdbf_code_t* code, const float* y_host,
                                            int64_t n_frames, float sigma, const ngdbf_params* params,
                                            uint64_t frame_offset, uint8_t* bits_host, int32_t* iters_host,
                                            uint8_t* pass_host, uint64_t* request_id) {
    if (!S || !code || !params) return fail(NGDBF_ERR_INVALID_ARG, "NULL server, code or params");
    ngdbf_status s = check_params(params, sigma);
    if (s != NGDBF_OK) return s;
    if (n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames >= (1ll << 31)) return fail(NGDBF_ERR_UNSUPPORTED, "a request holds fewer than 2^31 frames");
    if (n_frames > 0 && (!y_host || !bits_host || !iters_host || !pass_host))
        return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    if (code->device != S->device) return fail(NGDBF_ERR_INVALID_ARG, "code tables belong to another device");
    Request* r = new (std::nothrow) Request;
    if (!r) return fail(NGDBF_ERR_OOM, "host allocation");
    r->job.code = code;
    r->job.n_frames = n_frames;
    r->job.sigma = sigma;
    r->job.params = *params;
    r->job.frame_offset = frame_offset;
    r->y_host = y_host;
    r->bits_host = bits_host;
    r->iters_host = iters_host;
    r->pass_host = pass_host;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        r->id = ++S->stats.submitted;
        r->t_submit = now_s();
        S->pending.push_back(r);
    }
    S->cv.notify_all();
    if (request_id) *request_id = r->id;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_server_poll(ngdbf_server_t* S, uint64_t* ids, double* latency_s, int32_t* status,
                                          int32_t capacity, int32_t* n_out) {
    if (!S || !n_out || capacity < 0) return fail(NGDBF_ERR_INVALID_ARG, "bad poll arguments");
    std::lock_guard<std::mutex> lk(S->mu);
    int32_t k = 0;
    while (k < capacity && !S->completed.empty()) {
        Request* r = S->completed.front();
        S->completed.erase(S->completed.begin());
        if (ids) ids[k] = r->id;
        if (latency_s) latency_s[k] = r->t_done - r->t_submit;
        if (status) status[k] = r->status;
        delete r;
        ++k;
    }
    *n_out = k;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_server_wait(ngdbf_server_t* S, double timeout_s) {
    if (!S) return fail(NGDBF_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    while (S->stats.completed < S->stats.submitted) {
        if (S->cv.wait_until(lk, until) == std::cv_status::timeout && S->stats.completed < S->stats.submitted)
            return fail(NGDBF_ERR_TIMEOUT, "server: requests still running at the timeout");
    }
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_server_get_stats(ngdbf_server_t* S, ngdbf_server_stats* out) {
    if (!S || !out) return fail(NGDBF_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->stats;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_server_destroy(ngdbf_server_t* S) {
    if (!S) return NGDBF_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        for (Request* r : S->pending) delete r;
        S->pending.clear();
    }
    S->cv.notify_all();
    if (S->worker.joinable()) S->worker.join();     // admitted requests finish first, the kernel idles out
    S->epoch_img[0] = S->epoch;                     // and any kernel left exits at once
    cudaMemcpyAsync(&S->d_ring->stop_epoch, &S->epoch_img[0], 4, cudaMemcpyHostToDevice, S->pub_stream);
    cudaStreamSynchronize(S->pub_stream);
    cudaStreamSynchronize(S->serve_stream);
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (Staging* sg : S->stages) staging_release(sg);     // every copy out of them has completed
    cudaStreamDestroy(S->serve_stream);
    cudaStreamDestroy(S->pub_stream);
    cudaEventDestroy(S->ev_kernel);
    cudaFree(S->d_ring);
    cudaFree(S->d_claim);
    cudaFree(S->d_done);
    cudaFree(S->d_retire);
    cudaFreeHost(S->stage);
    cudaFreeHost(S->head_img);
    cudaFreeHost(S->epoch_img);
    cudaFreeHost(S->notify_host);
    for (Request* r : S->completed) delete r;
    delete S;
    return NGDBF_OK;
}
