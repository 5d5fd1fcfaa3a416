// ngdbf_device.cuh -- device-side arithmetic of the NGDBF decoder (sm_103a).
//
// Everything here is evaluated with explicitly rounded IEEE FP32 intrinsics
// (__fadd_rn, __fmul_rn, __fmaf_rn), so the compiler
// cannot contract or reassociate it: the perturbation q_k and the inversion
// function E_k of a frame are bit-identical wherever and however the frame
// is scheduled.
#pragma once

#include <cstdint>

namespace ngdbf {

// Constants of the Gaussian generator and of one decode, passed by value as
// kernel parameters (they live in the constant bank).
struct GenConsts {
    // Philox4x32-10 round keys: key + r * (0x9E3779B9, 0xBB67AE85), r = 0..9.
    uint32_t rk0[10];
    uint32_t rk1[10];
    // Inverse normal CDF: cubic coefficients (c0, c1, c2, c3) of segment 8 j + s,
    // level j = leading zeros of a = 2 (r mod 2^31) + 1, sub-interval s = the three
    // bits after a's leading one (see gauss_icdf).
    float4 icdf[256];
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the Weyl-bumped key xor-ed into the high halves.  Each product
// is formed as one 64-bit multiply, whose halves are the round's outputs.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const GenConsts& G, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0, p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t lo0 = (uint32_t)p0, hi0 = (uint32_t)(p0 >> 32);
        const uint32_t lo1 = (uint32_t)p1, hi1 = (uint32_t)(p1 >> 32);
        const uint32_t n0 = hi1 ^ c1 ^ G.rk0[r];
        const uint32_t n2 = hi0 ^ c3 ^ G.rk1[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// Standard normal deviate of one Philox output r by inversion of the normal CDF.
// Bit 31 of r is the sign; a = 2 (r mod 2^31) + 1 gives the lower-tail probability
// p = a 2^-33 in (0, 1/2).  With j = clz(a) and m = a << j, p lies in the j-th dyadic
// interval below 1/2, bits 30..28 of m pick one of its eight equal sub-intervals and
// bits 27..5 the position v in [-1/2, 1/2) inside it (exact in FP32), so that
// p = (8 + s + 1/2 + v) 2^-(j+5).  Phi^{-1}(p) is the segment's cubic in v (entry 8 j + s
// of tab, in shared memory), evaluated by Horner's rule with fused multiply-adds.
__device__ __forceinline__ float gauss_icdf(uint32_t r, const float4* tab) {
    const uint32_t a = (r << 1) | 1u;
    const uint32_t j = (uint32_t)__clz((int)a);
    const uint32_t m = a << j;
    const float4 c = tab[(j << 3) | ((m >> 28) & 7u)];
    const float v = __fadd_rn(__uint_as_float(0x3F800000u | ((m >> 5) & 0x007FFFFFu)), -1.5f);
    const float g = __fmaf_rn(__fmaf_rn(__fmaf_rn(c.w, v, c.z), v, c.y), v, c.x);
    return __uint_as_float(__float_as_uint(g) ^ (r & 0x80000000u));
}

// Uniform deviate on (-1, 1) of one Philox output (Sec. V-B variant): the top 24 bits a give
// the odd integer 2a + 1 - 2^24, exact in FP32, scaled by 2^-24 (exact).
__device__ __forceinline__ float uniform_dev(uint32_t r) {
    const int32_t odd = (int32_t)(2u * (r >> 8) + 1u) - (1 << 24);
    return __fmul_rn(__int2float_rn(odd), 5.9604644775390625e-08f);
}

// Four deviates for symbols 4g .. 4g+3 of frame (flo, fhi) at iteration t: symbol 4g + i takes
// Philox output i of counter (g, t, flo, fhi), as a standard normal deviate or, when `uniform`
// is set, as a uniform deviate on (-1, 1).
__device__ __forceinline__ void noise4(uint32_t g, uint32_t t, uint32_t flo, uint32_t fhi,
                                       const GenConsts& G, const float4* tab, bool uniform, float z[4]) {
    uint32_t r[4];
    philox4x32_10(g, t, flo, fhi, G, r);
    if (uniform) {
#pragma unroll
        for (int i = 0; i < 4; ++i) z[i] = uniform_dev(r[i]);
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) z[i] = gauss_icdf(r[i], tab);
    }
}

}  // namespace ngdbf
