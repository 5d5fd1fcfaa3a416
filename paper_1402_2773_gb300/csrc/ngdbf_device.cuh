// ngdbf_device.cuh -- device-side arithmetic of the NGDBF decoder (sm_103a).
//
// Everything here is evaluated with explicitly rounded IEEE FP32 intrinsics
// (__fadd_rn, __fmul_rn, __fmaf_rn, __fdiv_rn, __fsqrt_rn), so the compiler
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
    // 1/(2j+1) for j = 1..5 (atanh series of ln), fl32 of the exact quotient.
    float atanh_c[5];
    // (-1)^j (pi/2)^(2j+1) / (2j+1)!, j = 0..5   (sin series)
    float sin_c[6];
    // (-1)^j (pi/2)^(2j) / (2j)!,     j = 1..6   (cos series, constant 1 apart)
    float cos_c[6];
};

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with the Weyl-bumped key xor-ed into the high halves.
__device__ __forceinline__ void philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                              const GenConsts& G, uint32_t out[4]) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ G.rk0[r];
        const uint32_t n2 = hi0 ^ c3 ^ G.rk1[r];
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

// ln(u) for a positive normal float: u = m 2^e, m folded into (1/sqrt2, sqrt2],
// ln m = 2 atanh(s) with s = (m - 1) / (m + 1) and the atanh series to s^11.
__device__ __forceinline__ float ln_series(float u, const GenConsts& G) {
    const uint32_t b = __float_as_uint(u);
    int e = (int)((b >> 23) & 0xFFu) - 127;
    float m = __uint_as_float((b & 0x007FFFFFu) | 0x3F800000u);
    if (m > 0x1.6a09e6p+0f) {            // fl32(sqrt 2)
        m = __fmul_rn(m, 0.5f);
        e += 1;
    }
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float z = __fmul_rn(s, s);
    float p = G.atanh_c[4];
    p = __fmaf_rn(p, z, G.atanh_c[3]);
    p = __fmaf_rn(p, z, G.atanh_c[2]);
    p = __fmaf_rn(p, z, G.atanh_c[1]);
    p = __fmaf_rn(p, z, G.atanh_c[0]);
    const float r = __fmaf_rn(__fmul_rn(s, z), p, s);
    return __fmaf_rn(__int2float_rn(e), 0x1.62e430p-1f /* fl32(ln 2) */, __fmul_rn(2.0f, r));
}

// (b + 1/2) 2^-(bits) for an integer b < 2^bits <= 2^23, exactly: the float
// with exponent 0 and mantissa b is 1 + b 2^-23, and subtracting 1 - 2^-24
// leaves (2b + 1) 2^-24 without rounding; scaling by 2^(23 - bits) is exact.
__device__ __forceinline__ float half_offset_fraction(uint32_t b) {
    return __fadd_rn(__uint_as_float(0x3F800000u | b), -0x1.fffffep-1f);
}

// sin and cos of 2 pi u, u = (a + 1/2) 2^-23 with a a 23-bit integer.
// 4u = quadrant + xi exactly, xi in [-1/2, 1/2]; the series are in xi^2.
__device__ __forceinline__ void sincos_2pi(uint32_t a, const GenConsts& G, float& sn, float& cs) {
    uint32_t quad = (a >> 21) & 3u;
    const uint32_t rem = a & 0x1FFFFFu;
    // v = (rem + 1/2) 2^-21 in (0, 1); above 1/2 it moves to the next quadrant as v - 1
    const float v = __fmul_rn(half_offset_fraction(rem), 4.0f);
    float xi = v;
    if (rem >= (1u << 20)) {
        xi = __fadd_rn(v, -1.0f);
        quad = (quad + 1u) & 3u;
    }
    const float xx = __fmul_rn(xi, xi);
    float ps = G.sin_c[5];
    ps = __fmaf_rn(ps, xx, G.sin_c[4]);
    ps = __fmaf_rn(ps, xx, G.sin_c[3]);
    ps = __fmaf_rn(ps, xx, G.sin_c[2]);
    ps = __fmaf_rn(ps, xx, G.sin_c[1]);
    ps = __fmaf_rn(ps, xx, G.sin_c[0]);
    const float S = __fmul_rn(xi, ps);
    float pc = G.cos_c[5];
    pc = __fmaf_rn(pc, xx, G.cos_c[4]);
    pc = __fmaf_rn(pc, xx, G.cos_c[3]);
    pc = __fmaf_rn(pc, xx, G.cos_c[2]);
    pc = __fmaf_rn(pc, xx, G.cos_c[1]);
    pc = __fmaf_rn(pc, xx, G.cos_c[0]);
    const float C = __fmaf_rn(xx, pc, 1.0f);
    // rotation by quad quarter turns: (sin, cos) = (S,C), (C,-S), (-S,-C), (-C,S)
    const float s_ = (quad & 1u) ? C : S;
    const float c_ = (quad & 1u) ? S : C;
    sn = (quad & 2u) ? -s_ : s_;
    cs = ((quad + 1u) & 2u) ? -c_ : c_;
}

// Four standard normals for symbols 4g .. 4g+3 of frame (flo, fhi) at iteration t.
__device__ __forceinline__ void gauss4(uint32_t g, uint32_t t, uint32_t flo, uint32_t fhi,
                                       const GenConsts& G, float z[4]) {
    uint32_t r[4];
    philox4x32_10(g, t, flo, fhi, G, r);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const float u0 = half_offset_fraction(r[2 * h] >> 9);      // ((r >> 9) + 1/2) 2^-23
        const float rho = __fsqrt_rn(__fmul_rn(-2.0f, ln_series(u0, G)));
        float sn, cs;
        sincos_2pi(r[2 * h + 1] >> 9, G, sn, cs);
        z[2 * h] = __fmul_rn(rho, cs);
        z[2 * h + 1] = __fmul_rn(rho, sn);
    }
}

// E_k = ((x_k y_k) + w S_k) + q_k, rounded after every operation (Sec. III-C, Step 2).
__device__ __forceinline__ float inversion_metric(bool x_negative, float y, int S, float w, float q) {
    const float xy = x_negative ? -y : y;
    return __fadd_rn(__fadd_rn(xy, __fmul_rn(w, __int2float_rn(S))), q);
}

}  // namespace ngdbf
