// ngdbf_plain.cu -- the plain per-iteration form of the decoder: one thread per (frame, check)
// and per (frame, four symbols), one byte per decision, three launches per iteration (Step 1
// syndromes; retirement of the frames that satisfy every check or reached T; Step 2 / Step 3b
// updates), no bit-slicing, no persistent slots.  It computes exactly what the persistent
// kernels compute (same perturbation stream, same FP32 operations) and is the baseline they are
// measured against.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <string>

#include "ngdbf_host.h"

namespace ngdbf {
namespace {

struct PlainArgs {
    int32_t n, m, dv_max, dc_max, t_max, t_smooth, adapt, smooth, uniform, nb;
    int64_t n_frames;
    uint64_t frame_offset;
    const uint16_t* chk_cols;   // [dc_max][m], padded with n
    const uint16_t* sym_chks;   // [n][dv_max], padded with m
    const float* y;             // [F][n]
    float w, scale, y_max;
    int32_t clamp;
    const uint32_t* thr;        // [t_max + 1] FP32 bits of theta lambda^u
    int8_t* x;                  // [F][n + 1] decisions +-1 (entry n: +1, the padding)
    int8_t* s;                  // [F][m + 1] syndromes +-1 (entry m: 0, the padding)
    uint16_t* u;                // [F][n] adaptation counters
    int16_t* X;                 // [F][n] smoothing sums
    uint32_t* unsat;            // [F] some check unsatisfied at this iteration
    uint8_t* active;            // [F]
    uint8_t* bits;
    int32_t* iters;
    uint8_t* pass;
    GenConsts G;
};

__device__ __forceinline__ float held_sample(const PlainArgs& A, int64_t f, int k) {
    float v = A.y[f * A.n + k];
    if (A.clamp) {
        if (v > A.y_max) v = A.y_max;
        if (v < -A.y_max) v = -A.y_max;
    }
    return v;
}

// x(0) = sign(y) on the saturated samples; counters cleared; every frame active.
__global__ void plain_init(const __grid_constant__ PlainArgs A) {
    const int64_t total = A.n_frames * (A.n + 1);
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / (A.n + 1);
        const int k = (int)(e - f * (A.n + 1));
        if (k == A.n) {
            A.x[e] = 1;
            A.active[f] = 1;
            A.s[f * (A.m + 1) + A.m] = 0;
            continue;
        }
        A.x[e] = held_sample(A, f, k) >= 0.0f ? 1 : -1;
        A.u[f * A.n + k] = 0;
        A.X[f * A.n + k] = 0;
    }
}

// Step 1: s_i = prod_{j in N(i)} x_j for every active frame; unsat[f] set when some s_i = -1.
__global__ void plain_syndromes(const __grid_constant__ PlainArgs A) {
    const int64_t total = A.n_frames * A.m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / A.m;
        const int i = (int)(e - f * A.m);
        if (!A.active[f]) continue;
        const int8_t* xf = A.x + f * (A.n + 1);
        int p = 1;
        for (int j = 0; j < A.dc_max; ++j) p *= xf[A.chk_cols[j * A.m + i]];
        A.s[f * (A.m + 1) + i] = (int8_t)p;
        if (p < 0) atomicOr(A.unsat + f, 1u);
    }
}

// Retirement at iteration t (one CTA per frame): a frame with every check satisfied outputs x,
// iters = t, pass = 1; at t = T the smoothing sum takes x(T) and the frame outputs sign(X) (a
// zero sum keeps x), iters = T, pass = 0.  Otherwise the window sum takes x(t) here too.
__global__ void plain_retire(const __grid_constant__ PlainArgs A, int t) {
    const int64_t f = blockIdx.x;
    if (f >= A.n_frames || !A.active[f]) return;
    const bool ok = A.unsat[f] == 0u;
    const bool last = t >= A.t_max;
    int8_t* xf = A.x + f * (A.n + 1);
    int16_t* Xf = A.X + f * A.n;
    const bool window = A.smooth && t >= A.t_smooth && !ok;
    if (window)
        for (int k = threadIdx.x; k < A.n; k += blockDim.x) Xf[k] += xf[k];
    if (ok || last) {
        __syncthreads();
        for (int b = threadIdx.x; b < A.nb; b += blockDim.x) {
            uint32_t byte = 0;
            for (int q = 0; q < 8; ++q) {
                const int k = 8 * b + q;
                if (k >= A.n) break;
                int v = xf[k];
                if (!ok && A.smooth) v = Xf[k] > 0 ? 1 : (Xf[k] < 0 ? -1 : v);
                if (v < 0) byte |= 1u << q;
            }
            A.bits[f * A.nb + b] = (uint8_t)byte;
        }
        if (threadIdx.x == 0) {
            A.iters[f] = ok ? t : A.t_max;
            A.pass[f] = ok ? 1 : 0;
        }
        __syncthreads();
        if (threadIdx.x == 0) A.active[f] = 0;
    }
}

// Step 2 and Step 3b at iteration t < T for the four symbols 4g .. 4g+3 of an active frame
// (E_k = ((x_k y_k) + w S_k) + q_k rounded after every operation; flip when E_k < theta
// lambda^u_k, else u_k += 1 with adaptation).  Clears unsat[f] for the next iteration.
__global__ void plain_update(const __grid_constant__ PlainArgs A, int t) {
    __shared__ float4 tab[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) tab[i] = A.G.icdf[i];
    __syncthreads();
    const int groups = (A.n + 3) >> 2;
    const int64_t total = A.n_frames * groups;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t f = e / groups;
        const int g = (int)(e - f * groups);
        if (!A.active[f]) continue;
        if (g == 0) A.unsat[f] = 0u;
        const uint64_t fid = A.frame_offset + (uint64_t)f;
        float z[4];
        noise4((uint32_t)g, (uint32_t)t, (uint32_t)fid, (uint32_t)(fid >> 32), A.G, tab, A.uniform != 0, z);
        int8_t* xf = A.x + f * (A.n + 1);
        const int8_t* sf = A.s + f * (A.m + 1);
        for (int j = 0; j < 4; ++j) {
            const int k = 4 * g + j;
            if (k >= A.n) break;
            int S = 0;
            for (int d = 0; d < A.dv_max; ++d) S += sf[A.sym_chks[k * A.dv_max + d]];
            const float yv = held_sample(A, f, k);
            const float xy = xf[k] > 0 ? yv : -yv;
            const float ws = __fmul_rn(A.w, __int2float_rn(S));
            const float q = __fmul_rn(A.scale, z[j]);
            const float E = __fadd_rn(__fadd_rn(xy, ws), q);
            uint16_t& u = A.u[f * A.n + k];
            const float th = __uint_as_float(A.thr[A.adapt ? u : 0]);
            if (E < th) xf[k] = (int8_t)-xf[k];
            else if (A.adapt) u = (uint16_t)(u + 1);
        }
    }
}

}  // namespace
}  // namespace ngdbf

using namespace ngdbf;
using namespace ngdbf::host;

extern "C" ngdbf_status ngdbf_decode_plain(const ngdbf_code_t* C, const float* y, int64_t n_frames, float sigma,
                                           const ngdbf_params* P, uint64_t seed, uint64_t frame_offset, uint8_t* bits,
                                           int32_t* iters, uint8_t* pass, void* stream_ptr) {
    cudaStream_t stream = static_cast<cudaStream_t>(stream_ptr);
    if (!C) return fail(NGDBF_ERR_INVALID_ARG, "code is NULL");
    ngdbf_status st = check_params(P, sigma);
    if (st != NGDBF_OK) return st;
    if (P->variant & NGDBF_SINGLE)
        return fail(NGDBF_ERR_UNSUPPORTED, "the plain per-iteration form has no single-bit variant");
    if (P->precision != NGDBF_FP32) return fail(NGDBF_ERR_UNSUPPORTED, "the plain per-iteration form is FP32 only");
    if (n_frames < 0) return fail(NGDBF_ERR_INVALID_ARG, "n_frames < 0");
    if (n_frames == 0) return NGDBF_OK;
    if (!y || !bits || !iters || !pass) return fail(NGDBF_ERR_INVALID_ARG, "NULL buffer");
    int dev = 0, sms = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e, "device query");
    if (dev != C->device) return fail(NGDBF_ERR_INVALID_ARG, "code tables belong to another device");
    for (const void* p : {(const void*)y, (const void*)bits, (const void*)iters, (const void*)pass}) {
        cudaPointerAttributes a;
        e = cudaPointerGetAttributes(&a, p);
        if (e != cudaSuccess || !(a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
            cudaGetLastError();
            return fail(NGDBF_ERR_INVALID_ARG, "y, bits, iters and pass must be device memory");
        }
    }
    const int64_t F = n_frames, n = C->n, m = C->m, T = P->t_max;
    const size_t b_x = align256((size_t)F * (n + 1)), b_s = align256((size_t)F * (m + 1));
    const size_t b_u = align256((size_t)F * n * 2), b_X = align256((size_t)F * n * 2);
    const size_t b_f = align256((size_t)F * 4), b_a = align256((size_t)F), b_t = align256((size_t)(T + 1) * 4);
    cudaMemPool_t pool;
    st = get_pool(dev, &pool);
    if (st != NGDBF_OK) return st;
    void* ws = nullptr;
    e = cudaMallocFromPoolAsync(&ws, b_x + b_s + b_u + b_X + b_f + b_a + b_t, pool, stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(e == cudaErrorMemoryAllocation ? NGDBF_ERR_OOM : NGDBF_ERR_CUDA, "plain decode scratch");
    }
    unsigned char* p = static_cast<unsigned char*>(ws);
    PlainArgs A;
    std::memset(&A, 0, sizeof(A));
    Job J;
    std::vector<uint32_t> thr((size_t)T + 1);
    fill_job(C, P, y, F, sigma, frame_offset, bits, iters, pass, nullptr, &J, thr.data());
    A.n = (int32_t)n; A.m = (int32_t)m; A.dv_max = C->dv_max; A.dc_max = C->dc_max; A.t_max = (int32_t)T;
    A.t_smooth = J.t_smooth;
    A.adapt = (P->variant & NGDBF_ADAPT) ? 1 : 0;
    A.smooth = (P->variant & NGDBF_SMOOTH) ? 1 : 0;
    A.uniform = J.uniform;
    A.nb = J.nb;
    A.n_frames = F;
    A.frame_offset = frame_offset;
    A.chk_cols = C->d_chk_cols;
    A.sym_chks = C->d_sym_chks;
    A.y = y;
    A.w = J.w; A.scale = J.scale; A.y_max = J.y_max; A.clamp = J.clamp;
    A.x = reinterpret_cast<int8_t*>(p); p += b_x;
    A.s = reinterpret_cast<int8_t*>(p); p += b_s;
    A.u = reinterpret_cast<uint16_t*>(p); p += b_u;
    A.X = reinterpret_cast<int16_t*>(p); p += b_X;
    A.unsat = reinterpret_cast<uint32_t*>(p); p += b_f;
    A.active = p; p += b_a;
    A.thr = reinterpret_cast<uint32_t*>(p);
    A.bits = bits; A.iters = iters; A.pass = pass;
    host_gen_consts(seed, A.G);
    const int grid = sms * 8;
    int launches = 0;
    e = cudaMemcpyAsync(const_cast<uint32_t*>(A.thr), thr.data(), thr.size() * 4, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(A.unsat, 0, (size_t)F * 4, stream);
    if (e == cudaSuccess) {
        plain_init<<<grid, 256, 0, stream>>>(A);
        ++launches;
        e = cudaGetLastError();
    }
    for (int t = 0; t <= T && e == cudaSuccess; ++t) {
        plain_syndromes<<<grid, 256, 0, stream>>>(A);
        plain_retire<<<(unsigned)F, 256, 0, stream>>>(A, t);
        launches += 2;
        if (t < T) {
            plain_update<<<grid, 256, 0, stream>>>(A, t);
            ++launches;
        }
        e = cudaGetLastError();
    }
    cudaError_t ef = cudaFreeAsync(ws, stream);
    if (e != cudaSuccess) return cuda_fail(e, "plain decode launch");
    if (ef != cudaSuccess) return cuda_fail(ef, "cudaFreeAsync");
    set_last_launch(grid, 256, 0, 0, 0, launches, sms);
    return NGDBF_OK;
}
