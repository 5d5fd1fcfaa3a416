// ngdbf_hostmem.cu -- page-locked host memory for the host-buffer entry points
// (ngdbf_decode_host, the server), backed by transparent huge pages where the system has them.
//
// A copy engine reading page-locked host memory translates every page it touches; with
// small pages scattered in physical memory (the first large allocation of a process often
// gets them) those translations miss and the copy runs at a tenth of the link rate.  Memory
// mapped on huge-page boundaries with MADV_HUGEPAGE and then registered with CUDA needs one
// translation per huge page, so copies from it stay at full rate.  Requests below one huge
// page, and systems where the mapping or registration fails, get cudaHostAlloc memory.
#include <cuda_runtime.h>
#include <sys/mman.h>

#include <cstdint>
#include <cstdio>
#include <map>
#include <mutex>

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

// Huge-page-aligned anonymous mapping of `len` bytes (a multiple of hp), advised for huge
// pages; nullptr on failure.
void* map_aligned(size_t len, size_t hp) {
    void* m = mmap(nullptr, len + hp, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
    if (m == MAP_FAILED) return nullptr;
    const uintptr_t base = reinterpret_cast<uintptr_t>(m);
    const uintptr_t start = (base + hp - 1) / hp * hp;
    if (start > base) munmap(m, start - base);
    const uintptr_t end = start + len, map_end = base + len + hp;
    if (map_end > end) munmap(reinterpret_cast<void*>(end), map_end - end);
    void* p = reinterpret_cast<void*>(start);
    madvise(p, len, MADV_HUGEPAGE);     // advice only: base pages when the system has no huge pages
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

extern "C" ngdbf_status ngdbf_host_huge_page_bytes(int64_t* out) {
    if (!out) return fail(NGDBF_ERR_INVALID_ARG, "out is NULL");
    *out = (int64_t)huge_page_bytes();
    return NGDBF_OK;
}
