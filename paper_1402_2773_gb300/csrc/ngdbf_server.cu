// ngdbf_server.cu -- the serving loop: a scheduler thread that admits decode requests
// under a device-memory budget and runs them as job-table launches on several streams.
//
// A launch holds, in one block from the library's stream-ordered pool:
//   [queues | job table | thresholds | first job per CTA | slot samples | slot state |
//    per request: samples, bits, iterations, pass flags]
// The job table, thresholds and first jobs are staged in page-locked host memory and
// copied with one asynchronous copy.  A host function enqueued after the output copies
// stamps the completion time and wakes the scheduler, which then frees the block.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "ngdbf_host.h"

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
};

struct Launch {
    std::vector<Request*> reqs;
    unsigned char* block = nullptr;  // device memory of the launch
    size_t bytes = 0;
    unsigned char* stage = nullptr;  // page-locked staging of the job table
    size_t stage_bytes = 0;
    int stream = -1;
    std::atomic<bool> done{false};
    double t_done = 0;
    void* server = nullptr;
};

}  // namespace

struct ngdbf_server {
    int device = 0;
    size_t budget = 0;
    int max_launches = 1, max_jobs = 1;
    uint64_t seed = 0;
    cudaMemPool_t pool = nullptr;
    std::vector<cudaStream_t> streams;
    std::vector<bool> stream_busy;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<Request*> pending;
    std::vector<Launch*> inflight;
    std::vector<Request*> completed;          // not yet reported by poll
    std::vector<std::pair<unsigned char*, size_t>> free_stage;
    size_t in_use = 0;
    uint64_t next_id = 1;
    ngdbf_server_stats stats{};
    bool stop = false;
    std::thread worker;
};

namespace {

void CUDART_CB launch_finished(void* arg) {
    Launch* L = static_cast<Launch*>(arg);
    // once `done` is set the scheduler may retire and delete L: read what is needed first.
    // The server outlives this call (ngdbf_server_destroy synchronizes the streams).
    ngdbf_server* S = static_cast<ngdbf_server*>(L->server);
    L->t_done = now_s();
    L->done.store(true);
    S->cv.notify_all();
}

// Device bytes of a request's own buffers.
size_t request_bytes(const ngdbf_job& q) {
    const int64_t n = q.code->n, nb = (n + 7) / 8;
    return align256((size_t)q.n_frames * n * 4) + align256((size_t)q.n_frames * nb) +
           align256((size_t)q.n_frames * 4) + align256((size_t)q.n_frames);
}

struct LaunchLayout {
    TablePlan plan;
    int grid = 0, block = 0;
    size_t off_jobs = 0, off_thr = 0, off_first = 0, off_y = 0, off_st = 0, off_req = 0, total = 0;
    size_t stage_bytes = 0;
};

// Plan and size one launch of the given requests (all of one variant and precision).
ngdbf_status layout_launch(ngdbf_server* S, const std::vector<Request*>& reqs, LaunchLayout* out) {
    std::vector<ngdbf_job> jobs;
    for (Request* r : reqs) jobs.push_back(r->job);
    LaunchLayout& L = *out;
    ngdbf_status s = plan_table(jobs.data(), (int32_t)jobs.size(), S->device, &L.plan);
    if (s != NGDBF_OK) return s;
    const int J = (int)reqs.size();
    int64_t groups = 0;
    for (const ngdbf_job& q : jobs) groups += (q.n_frames + 31) / 32;
    L.block = L.plan.shapes[0].first;
    L.grid = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)L.plan.sm_count * L.plan.shapes[0].second, groups));
    const size_t per_slot_y = (size_t)pad4(L.plan.n_max) * kSlots * held_bytes(L.plan.precision);
    const size_t per_slot_st = L.plan.state_global ? (size_t)pad4(L.plan.n_max) * kSlots * 2 : 0;
    L.off_jobs = align256(8 * (size_t)J);                 // queues first
    L.off_thr = L.off_jobs + align256(sizeof(Job) * J);
    L.off_first = L.off_thr + align256(L.plan.thr_words * 4);
    L.off_y = L.off_first + align256(4 * (size_t)L.grid);
    L.off_st = L.off_y + align256((size_t)L.grid * per_slot_y);
    L.off_req = L.off_st + align256((size_t)L.grid * per_slot_st);
    L.total = L.off_req;
    for (const ngdbf_job& q : jobs) L.total += request_bytes(q);
    L.stage_bytes = L.off_y - L.off_jobs;                   // job table, thresholds, first jobs
    return NGDBF_OK;
}

unsigned char* take_stage(ngdbf_server* S, size_t bytes, size_t* got) {
    for (size_t i = 0; i < S->free_stage.size(); ++i)
        if (S->free_stage[i].second >= bytes) {
            auto e = S->free_stage[i];
            S->free_stage.erase(S->free_stage.begin() + i);
            *got = e.second;
            return e.first;
        }
    void* p = nullptr;
    const size_t sz = std::max<size_t>(bytes, 1 << 16);
    if (cudaMallocHost(&p, sz) != cudaSuccess) return nullptr;
    *got = sz;
    return static_cast<unsigned char*>(p);
}

// Issues copy-in, decode and copy-out of one admitted launch on stream `si`.
ngdbf_status issue(ngdbf_server* S, Launch* Lc, const LaunchLayout& L, int si) {
    cudaStream_t st = S->streams[si];
    cudaError_t e = cudaMallocFromPoolAsync(reinterpret_cast<void**>(&Lc->block), L.total, S->pool, st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(NGDBF_ERR_OOM, "server: device block"); }
    Lc->bytes = L.total;
    Lc->stage = take_stage(S, L.stage_bytes, &Lc->stage_bytes);
    if (!Lc->stage) return fail(NGDBF_ERR_OOM, "server: staging");
    unsigned char* base = Lc->block;
    const int J = (int)Lc->reqs.size();
    std::vector<int64_t> frames(J), weight(J);
    Job* hjobs = reinterpret_cast<Job*>(Lc->stage);
    uint32_t* hthr = reinterpret_cast<uint32_t*>(Lc->stage + (L.off_thr - L.off_jobs));
    int32_t* hfirst = reinterpret_cast<int32_t*>(Lc->stage + (L.off_first - L.off_jobs));
    size_t pos = L.off_req, tpos = 0;
    for (int j = 0; j < J; ++j) {
        Request* r = Lc->reqs[j];
        const ngdbf_job& q = r->job;
        const int64_t n = q.code->n, nb = (n + 7) / 8, F = q.n_frames;
        float* dy = reinterpret_cast<float*>(base + pos);
        pos += align256((size_t)F * n * 4);
        uint8_t* dbits = base + pos;
        pos += align256((size_t)F * nb);
        int32_t* diters = reinterpret_cast<int32_t*>(base + pos);
        pos += align256((size_t)F * 4);
        uint8_t* dpass = base + pos;
        pos += align256((size_t)F);
        fill_job(q.code, &q.params, dy, F, q.sigma, q.frame_offset, dbits, diters, dpass,
                 reinterpret_cast<unsigned long long*>(base) + j, &hjobs[j], hthr + tpos);
        hjobs[j].thr = reinterpret_cast<const uint32_t*>(base + L.off_thr) + tpos;
        tpos += (size_t)q.params.t_max + 1;
        frames[j] = F;
        weight[j] = F * n * (q.params.t_max + 1);
        if (F > 0) {
            e = cudaMemcpyAsync(dy, r->y_host, (size_t)F * n * 4, cudaMemcpyHostToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e, "server: copy in");
        }
    }
    std::vector<int32_t> first = assign_ctas(frames, weight, L.grid);
    std::memcpy(hfirst, first.data(), first.size() * 4);
    e = cudaMemcpyAsync(base + L.off_jobs, Lc->stage, L.stage_bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(base, 0, 8 * (size_t)J, st);
    if (e != cudaSuccess) return cuda_fail(e, "server: job table");
    MultiArgs A;
    std::memset(&A, 0, sizeof(A));
    A.jobs = reinterpret_cast<const Job*>(base + L.off_jobs);
    A.n_jobs = J;
    A.first_job = reinterpret_cast<const int32_t*>(base + L.off_first);
    A.n_max = L.plan.n_max; A.m_max = L.plan.m_max; A.t_max = L.plan.t_max;
    A.dv_max = L.plan.dv_max; A.dc_max = L.plan.dc_max;
    A.placement = L.plan.placement;
    A.yslots = base + L.off_y;
    A.st_global = L.plan.state_global ? reinterpret_cast<uint16_t*>(base + L.off_st) : nullptr;
    host_gen_consts(S->seed, A.G);
    e = launch_multi(L.plan.fn, A, L.grid, L.block, L.plan.smem, st);
    if (e != cudaSuccess) return cuda_fail(e, "server: launch");
    for (int j = 0; j < J; ++j) {
        Request* r = Lc->reqs[j];
        const Job& hj = hjobs[j];
        const int64_t F = r->job.n_frames, nb = (r->job.code->n + 7) / 8;
        if (F == 0) continue;
        e = cudaMemcpyAsync(r->bits_host, hj.bits, (size_t)F * nb, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->iters_host, hj.iters, (size_t)F * 4, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(r->pass_host, hj.pass, (size_t)F, cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return cuda_fail(e, "server: copy out");
    }
    Lc->stream = si;
    Lc->server = S;
    e = cudaLaunchHostFunc(st, launch_finished, Lc);
    if (e != cudaSuccess) return cuda_fail(e, "server: completion callback");
    return NGDBF_OK;
}

void finish_requests(ngdbf_server* S, const std::vector<Request*>& reqs, double t, int32_t status) {
    for (Request* r : reqs) {
        r->t_done = t;
        r->status = status;
        S->completed.push_back(r);
        S->stats.completed += 1;
        if (status != NGDBF_OK) S->stats.failed += 1;
        else S->stats.frames += r->job.n_frames;
    }
}

void scheduler(ngdbf_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // requests completed or launches issued in this pass: waiters are woken after it
        // (ngdbf_server_wait sleeps on the same condition until every request completed)
        bool progressed = false;
        // retire finished launches
        for (size_t i = 0; i < S->inflight.size();) {
            Launch* L = S->inflight[i];
            if (!L->done.load()) { ++i; continue; }
            cudaFreeAsync(L->block, S->streams[L->stream]);
            S->free_stage.push_back({L->stage, L->stage_bytes});
            S->in_use -= L->bytes;
            S->stream_busy[L->stream] = false;
            finish_requests(S, L->reqs, L->t_done, NGDBF_OK);
            delete L;
            S->inflight.erase(S->inflight.begin() + i);
            progressed = true;
        }
        // admit pending requests in arrival order into one launch per free stream
        while (!S->pending.empty() && !S->stop) {
            int si = -1;
            for (int k = 0; k < (int)S->streams.size(); ++k)
                if (!S->stream_busy[k]) { si = k; break; }
            if (si < 0) break;
            std::vector<Request*> group;
            LaunchLayout L;
            const int variant = S->pending.front()->job.params.variant;
            const int precision = S->pending.front()->job.params.precision;
            for (Request* r : S->pending) {
                if ((int)group.size() >= S->max_jobs) break;
                if (r->job.params.variant != variant || r->job.params.precision != precision) break;
                group.push_back(r);
                LaunchLayout trial;
                if (layout_launch(S, group, &trial) != NGDBF_OK || S->in_use + trial.total > S->budget) {
                    group.pop_back();
                    break;
                }
                L = trial;
            }
            if (group.empty()) {
                Request* r = S->pending.front();
                LaunchLayout alone;
                ngdbf_status s = layout_launch(S, {r}, &alone);
                if (s != NGDBF_OK || (alone.total > S->budget)) {
                    // can never run: report it and go on
                    S->pending.pop_front();
                    finish_requests(S, {r}, now_s(), s != NGDBF_OK ? s : NGDBF_ERR_OOM);
                    progressed = true;
                    continue;
                }
                break;                       // wait for memory to be returned
            }
            for (size_t k = 0; k < group.size(); ++k) S->pending.pop_front();
            Launch* Lc = new Launch;
            Lc->reqs = group;
            S->stream_busy[si] = true;
            ngdbf_status s = issue(S, Lc, L, si);
            if (s != NGDBF_OK) {
                cudaStreamSynchronize(S->streams[si]);
                if (Lc->block) cudaFreeAsync(Lc->block, S->streams[si]);
                if (Lc->stage) S->free_stage.push_back({Lc->stage, Lc->stage_bytes});
                S->stream_busy[si] = false;
                finish_requests(S, group, now_s(), s);
                delete Lc;
            } else {
                S->in_use += L.total;
                S->inflight.push_back(Lc);
                S->stats.launches += 1;
                S->stats.peak_bytes_in_use = std::max<int64_t>(S->stats.peak_bytes_in_use, (int64_t)S->in_use);
                S->stats.peak_concurrent_launches =
                    std::max<int32_t>(S->stats.peak_concurrent_launches, (int32_t)S->inflight.size());
            }
            progressed = true;
        }
        if (progressed) S->cv.notify_all();
        if (S->stop && S->inflight.empty()) break;
        S->cv.wait_for(lk, std::chrono::microseconds(200));
    }
}

}  // namespace

extern "C" ngdbf_status ngdbf_server_create(size_t device_budget_bytes, int32_t max_inflight_launches,
                                            int32_t max_jobs_per_launch, uint64_t seed, ngdbf_server_t** out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (device_budget_bytes == 0) return fail(NGDBF_ERR_INVALID_ARG, "budget must be > 0");
    if (max_inflight_launches < 1 || max_inflight_launches > 16)
        return fail(NGDBF_ERR_INVALID_ARG, "max_inflight_launches must be 1..16");
    if (max_jobs_per_launch < 1 || max_jobs_per_launch > 4096)
        return fail(NGDBF_ERR_INVALID_ARG, "max_jobs_per_launch must be 1..4096");
    ngdbf_server* S = new (std::nothrow) ngdbf_server;
    if (!S) return fail(NGDBF_ERR_OOM, "host allocation");
    cudaError_t e = cudaGetDevice(&S->device);
    if (e != cudaSuccess) { delete S; return cuda_fail(e, "cudaGetDevice"); }
    ngdbf_status s = get_pool(S->device, &S->pool);
    if (s != NGDBF_OK) { delete S; return s; }
    S->budget = device_budget_bytes;
    S->max_launches = max_inflight_launches;
    S->max_jobs = max_jobs_per_launch;
    S->seed = seed;
    for (int k = 0; k < max_inflight_launches; ++k) {
        cudaStream_t st;
        e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (cudaStream_t t : S->streams) cudaStreamDestroy(t);
            delete S;
            return cuda_fail(e, "server streams");
        }
        S->streams.push_back(st);
        S->stream_busy.push_back(false);
    }
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
        r->id = S->next_id++;
        r->t_submit = now_s();
        S->pending.push_back(r);
        S->stats.submitted += 1;
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
    if (S->worker.joinable()) S->worker.join();
    for (cudaStream_t st : S->streams) {
        cudaStreamSynchronize(st);
        cudaStreamDestroy(st);
    }
    for (auto& b : S->free_stage) cudaFreeHost(b.first);
    for (Request* r : S->completed) delete r;
    delete S;
    return NGDBF_OK;
}
