// ngdbf_hostmem.cu -- page-locked host memory for the host-buffer entry points
// (ngdbf_decode_host, the server), backed by transparent huge pages where the system has them.
//
// Blocks of at least one transparent huge page are mapped on huge-page boundaries, advised
// for huge pages (one translation per huge page where the kernel can back them) and registered
// with CUDA; ngdbf_host_block_info reports how much of a block the kernel backs with huge
// pages.  Requests below one huge page, and systems where the mapping or registration fails,
// get cudaHostAlloc memory.
#include <cuda_runtime.h>
#include <sys/mman.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "ngdbf_host.h"

using namespace ngdbf::host;

namespace {

struct HostBlock {
    size_t length;      // bytes mapped (a multiple of the huge-page size); 0: cudaHostAlloc memory
};

std::mutex g_host_mu;
std::map<uintptr_t, HostBlock> g_host_blocks;

// Size of a PMD-level transparent huge page (2 MiB with 4 KiB base pages, 512 MiB with
// 64 KiB base pages); 0 when the system does not report one.
size_t huge_page_bytes() {
    static const size_t hp = [] {
        unsigned long long v = 0;
        if (FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
            if (std::fscanf(f, "%llu", &v) != 1) v = 0;
            std::fclose(f);
        }
        return (size_t)v;
    }();
    return hp;
}

// Huge-page-aligned anonymous mapping of `len` bytes (a multiple of hp); nullptr on failure.
void* map_aligned(size_t len, size_t hp) {
    void* m = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED) return nullptr;
    const uintptr_t base = reinterpret_cast<uintptr_t>(m);
    const uintptr_t start = (base + hp - 1) / hp * hp;
    if (start > base) munmap(m, start - base);
    const uintptr_t end = start + len, map_end = base + len + hp;
    if (map_end > end) munmap(reinterpret_cast<void*>(end), map_end - end);
    void* p = reinterpret_cast<void*>(start);
    madvise(p, len, MADV_HUGEPAGE);
    return p;
}

}  // namespace

extern "C" ngdbf_status ngdbf_host_alloc(size_t bytes, void** out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (bytes == 0) return fail(NGDBF_ERR_INVALID_ARG, "bytes == 0");
    const size_t hp = huge_page_bytes();
    void* p = nullptr;
    size_t length = 0;
    if (hp > 0 && bytes >= hp && bytes <= SIZE_MAX - 2 * hp) {
        const size_t len = (bytes + hp - 1) / hp * hp;
        p = map_aligned(len, hp);
        if (p) {
            if (cudaHostRegister(p, len, cudaHostRegisterDefault) == cudaSuccess) {
                length = len;
            } else {
                cudaGetLastError();
                munmap(p, len);
                p = nullptr;
            }
        }
    }
    if (!p) {
        cudaError_t e = cudaHostAlloc(&p, bytes, cudaHostAllocDefault);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(e == cudaErrorMemoryAllocation ? NGDBF_ERR_OOM : NGDBF_ERR_CUDA,
                        std::string("page-locked host allocation: ") + cudaGetErrorString(e));
        }
    }
    std::lock_guard<std::mutex> g(g_host_mu);
    g_host_blocks[reinterpret_cast<uintptr_t>(p)] = HostBlock{length};
    *out = p;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_host_free(void* p) {
    if (!p) return NGDBF_OK;
    HostBlock b;
    {
        std::lock_guard<std::mutex> g(g_host_mu);
        auto it = g_host_blocks.find(reinterpret_cast<uintptr_t>(p));
        if (it == g_host_blocks.end()) return fail(NGDBF_ERR_INVALID_ARG, "pointer not from ngdbf_host_alloc");
        b = it->second;
        g_host_blocks.erase(it);
    }
    if (b.length == 0) {
        cudaError_t e = cudaFreeHost(p);
        if (e != cudaSuccess) return cuda_fail(e, "cudaFreeHost");
        return NGDBF_OK;
    }
    cudaError_t e = cudaHostUnregister(p);
    munmap(p, b.length);
    if (e != cudaSuccess) return cuda_fail(e, "cudaHostUnregister");
    return NGDBF_OK;
}

// Bytes of [p, p + len) that the kernel backs with transparent huge pages, from the
// AnonHugePages lines of /proc/self/smaps for the mappings that overlap the range (a mapping
// only partly inside the range counts in proportion); -1 when smaps cannot be read.
static int64_t huge_backed_bytes(uintptr_t p, size_t len) {
    FILE* f = std::fopen("/proc/self/smaps", "r");
    if (!f) return -1;
    char line[512];
    int64_t total = 0;
    unsigned long long lo = 0, hi = 0;
    bool in = false;
    while (std::fgets(line, sizeof(line), f)) {
        unsigned long long a = 0, b = 0;
        char perms[8];
        if (std::sscanf(line, "%llx-%llx %7s", &a, &b, perms) == 3) {
            lo = a;
            hi = b;
            in = hi > p && lo < p + len;
            continue;
        }
        unsigned long long kb = 0;
        if (in && std::sscanf(line, "AnonHugePages: %llu kB", &kb) == 1) {
            const unsigned long long s = std::max<unsigned long long>(lo, p);
            const unsigned long long e = std::min<unsigned long long>(hi, p + len);
            const double part = (double)(e - s) / (double)(hi - lo);
            total += (int64_t)((double)kb * 1024.0 * part);
        }
    }
    std::fclose(f);
    return total;
}

extern "C" ngdbf_status ngdbf_host_block_info(const void* p, int64_t* bytes, int64_t* huge_bytes) {
    if (!p || !bytes || !huge_bytes) return fail(NGDBF_ERR_INVALID_ARG, "NULL argument");
    size_t len = 0;
    {
        std::lock_guard<std::mutex> g(g_host_mu);
        auto it = g_host_blocks.find(reinterpret_cast<uintptr_t>(p));
        if (it == g_host_blocks.end()) return fail(NGDBF_ERR_INVALID_ARG, "pointer not from ngdbf_host_alloc");
        len = it->second.length;
    }
    *bytes = (int64_t)len;
    *huge_bytes = len ? huge_backed_bytes(reinterpret_cast<uintptr_t>(p), len) : 0;
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_host_huge_page_bytes(int64_t* out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = (int64_t)huge_page_bytes();
    return NGDBF_OK;
}

// ---------------------------------------------------------------------------
// Staged host-to-device copies for ngdbf_decode_host: the host threads of a small pool copy
// the caller's samples into one of two page-locked staging buffers that the library keeps
// and reuses (so the copy engines' translations of them stay cached), and the device copies
// from there.  On the GB300 hosts measured, direct copies from the first several GB of
// page-locked memory a process registered ran at 2-20 GB/s when cold, against 210 GB/s from
// the rest; staged copies run at the host's memcpy rate (about 120 GB/s with 16 threads)
// whatever the caller's buffer is, page-locked or not.
// ---------------------------------------------------------------------------

namespace {

// Fixed pool of host threads that split one memcpy between them.
class CopyPool {
  public:
    explicit CopyPool(int n) : n_(n) {
        for (int i = 1; i < n_; ++i) th_.emplace_back([this, i] { run(i); });
    }
    ~CopyPool() {
        {
            std::lock_guard<std::mutex> g(mu_);
            stop_ = true;
            ++gen_;
        }
        cv_.notify_all();
        for (auto& t : th_) t.join();
    }
    // Copies `bytes` from src to dst, the calling thread taking the first share.
    void copy(void* dst, const void* src, size_t bytes) {
        std::unique_lock<std::mutex> lk(call_mu_);
        {
            std::lock_guard<std::mutex> g(mu_);
            dst_ = static_cast<unsigned char*>(dst);
            src_ = static_cast<const unsigned char*>(src);
            bytes_ = bytes;
            pending_ = n_ - 1;
            ++gen_;
        }
        cv_.notify_all();
        part(0);
        std::unique_lock<std::mutex> g(mu_);
        done_cv_.wait(g, [this] { return pending_ == 0; });
    }

  private:
    void part(int i) {
        // shares of whole 4 KiB pages, the last share takes the remainder
        const size_t pages = bytes_ / 4096, per = pages / (size_t)n_;
        const size_t lo = (size_t)i * per * 4096;
        const size_t hi = i == n_ - 1 ? bytes_ : (size_t)(i + 1) * per * 4096;
        if (hi > lo) std::memcpy(dst_ + lo, src_ + lo, hi - lo);
    }
    void run(int i) {
        unsigned long long seen = 0;
        for (;;) {
            {
                std::unique_lock<std::mutex> g(mu_);
                cv_.wait(g, [&] { return gen_ != seen; });
                seen = gen_;
                if (stop_) return;
            }
            part(i);
            {
                std::lock_guard<std::mutex> g(mu_);
                if (--pending_ == 0) done_cv_.notify_one();
            }
        }
    }
    int n_;
    std::vector<std::thread> th_;
    std::mutex mu_, call_mu_;
    std::condition_variable cv_, done_cv_;
    unsigned char* dst_ = nullptr;
    const unsigned char* src_ = nullptr;
    size_t bytes_ = 0;
    int pending_ = 0;
    unsigned long long gen_ = 0;
    bool stop_ = false;
};

CopyPool& copy_pool() {
    static CopyPool pool([] {
        const unsigned hw = std::thread::hardware_concurrency();
        return (int)std::max(1u, std::min(16u, hw ? hw : 1u));
    }());
    return pool;
}

std::atomic<int> g_copy_mode{NGDBF_HOST_COPY_STAGED};

}  // namespace

namespace ngdbf {
namespace host {

struct Staging {
    int device = -1;
    unsigned char* buf[2] = {nullptr, nullptr};
    cudaEvent_t free_ev[2] = {nullptr, nullptr};     // recorded after the copy out of buf[k]
    int next = 0;
};

namespace {
std::mutex g_stage_mu;
std::vector<Staging*> g_stage_free;
void staging_destroy(Staging* s) {
    for (int k = 0; k < 2; ++k) {
        if (s->free_ev[k]) cudaEventDestroy(s->free_ev[k]);
        if (s->buf[k]) cudaFreeHost(s->buf[k]);
    }
    delete s;
}
}  // namespace

int host_copy_mode() { return g_copy_mode.load(); }

Staging* staging_acquire(int dev) {
    {
        std::lock_guard<std::mutex> g(g_stage_mu);
        for (size_t i = 0; i < g_stage_free.size(); ++i) {
            if (g_stage_free[i]->device != dev) continue;
            Staging* s = g_stage_free[i];
            g_stage_free.erase(g_stage_free.begin() + i);
            return s;
        }
    }
    Staging* s = new (std::nothrow) Staging;
    if (!s) return nullptr;
    s->device = dev;
    bool ok = true;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaHostAlloc(reinterpret_cast<void**>(&s->buf[k]), kStageBytes, cudaHostAllocDefault) == cudaSuccess &&
             cudaEventCreateWithFlags(&s->free_ev[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        staging_destroy(s);
        return nullptr;
    }
    return s;
}

void staging_release(Staging* s) {
    if (!s) return;
    std::lock_guard<std::mutex> g(g_stage_mu);
    g_stage_free.push_back(s);
}

cudaError_t staged_h2d(Staging* s, void* dst, const void* src, size_t bytes, cudaStream_t st) {
    for (size_t off = 0; off < bytes; off += kStageBytes) {
        const size_t len = std::min(kStageBytes, bytes - off);
        const int k = s->next;
        s->next ^= 1;
        cudaError_t e = cudaEventSynchronize(s->free_ev[k]);    // the last copy out of buf[k] is done
        if (e != cudaSuccess) return e;
        copy_pool().copy(s->buf[k], static_cast<const unsigned char*>(src) + off, len);
        e = cudaMemcpyAsync(static_cast<unsigned char*>(dst) + off, s->buf[k], len, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = cudaEventRecord(s->free_ev[k], st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace host
}  // namespace ngdbf

extern "C" ngdbf_status ngdbf_set_host_copy_mode(int32_t mode) {
    if (mode != NGDBF_HOST_COPY_STAGED && mode != NGDBF_HOST_COPY_DIRECT)
        return fail(NGDBF_ERR_INVALID_ARG, "unknown host copy mode");
    g_copy_mode.store(mode);
    return NGDBF_OK;
}

extern "C" ngdbf_status ngdbf_get_host_copy_mode(int32_t* mode) {
    if (!mode) return fail(NGDBF_ERR_INVALID_ARG, "mode is NULL");
    *mode = g_copy_mode.load();
    return NGDBF_OK;
}
