/*
 * ngdbf_oracle.c -- reference NGDBF decoder.  TEST INFRASTRUCTURE ONLY.
 *
 * This file is the plain, slow, step-by-step statement of Noisy Gradient
 * Descent Bit-Flip decoding (Sundararajan, Winstead, Boutillon, "Noisy
 * Gradient Descent Bit-Flip Decoding for LDPC Codes", IEEE Trans. Commun.
 * 2014).  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code with the CUDA decoder.
 *
 * Paper sections followed:
 *   Sec. III-A  notation: H, N(i), M(k), x(0) = sign(y), bipolar syndromes
 *   Sec. III-B  GDBF Steps 1-4 (Step 1 syndrome + stop, Step 3b multi-bit flip,
 *               Step 3a single-bit flip of argmin E_k for S-NGDBF)
 *   Sec. III-C  NGDBF Step 2: E_k = x_k y_k + w sum_{i in M(k)} s_i + q_k,
 *               q_k ~ N(0, eta^2 N0/2)
 *   Sec. III-D  threshold adaptation Steps 0 and 3b (theta_k <- theta_k lambda
 *               when not flipped), in the counter form of Sec. V-A,
 *               theta_k = theta lambda^{u_k} (Eqs. 11-12)
 *   Sec. III-E  output smoothing, Eq. 7: X_k(t+1) = X_k(t) + x_k(t) over
 *               t = T-W .. T, output sign(X_k) when T is reached
 *   Sec. IV-E   quantizer g(.) (Eq. 8)
 *   Sec. V-A    quantized threshold adaptation events (Eq. 13, Table II)
 *
 * Readings where the paper is silent (each also listed in the design notes):
 *   - sign(0) = +1; samples are clamped to [-Y_max, Y_max] first (Sec. IV-A).
 *   - Step 1 precedes Step 2; a frame valid at t reports iters = t, pass = 1;
 *     T flip phases at most, iters = T and pass = 0 when T is reached.
 *   - Flooding schedule: every E_k of iteration t uses the syndromes of t.
 *   - Strict E_k < theta_k flips; a tie adapts (u_k += 1).
 *   - Single-bit (Step 3a): the flipped symbol is the first k with the least
 *     E_k (ties go to the lowest index); no threshold, no adaptation.
 *   - The smoothing sum covers x(t) for t = max(0, T-W) .. T; a zero sum keeps
 *     x_k(T).
 *   - Perturbation std = eta * sigma with sigma the channel std (N0/2 = sigma^2).
 *   - The quantizer's level index saturates at 2^(Q-1) - 1 (needed to
 *     reproduce Table II).
 *
 * The perturbation q_k is drawn by a counter-based generator (the paper's own
 * hardware used one Gaussian RNG and a shift-register chain, Sec. V-B):
 *   Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), key = (seed_lo,
 *   seed_hi), counter = (k/4, t, frame_lo, frame_hi); output k mod 4 gives
 *   q_k's standard normal deviate by inversion of the normal CDF (below).
 * The FP32 form replaces Phi^{-1} by piecewise cubics with a fixed table, so
 * that the same definition can be evaluated bit-identically elsewhere; the
 * FP64 form refines it to double accuracy with the C library's erfc.
 *
 * Reduced-precision forms of the inversion function (Sec. IV-E), on the same
 * FP32 perturbation q_k:
 *   FP16:  y, w, q and theta lambda^u rounded to binary16 (nearest-even);
 *          E = h(h(x y + h(w S)) + q) with h() rounding each FP32 result to
 *          binary16 (one FP32 operation on binary16 operands, then one
 *          rounding, is the correctly rounded binary16 operation); S is an
 *          exact integer.
 *   FIX:   Eq. 8 with Q bits: level k = min(floor(|v| R), 2^(Q-1) - 1) with
 *          R = fl32(2^Q / (2 Y_max)) and the product |v| R in FP32; held as the
 *          signed code b = k (v >= 0) or -k-1 (v < 0), value 2b + 1 in units of
 *          Delta/2 = Y_max / 2^Q.  E~ = x Y~ + W~ S + Q~ in exact integers,
 *          compared with Theta~(u) = value of fl32(theta lambda^u).
 *   FIXACC: the held sample is the Eq. 8 level code of y (Q bits) exactly as in
 *          FIX, but the inversion function is accumulated in exact int32 in a
 *          finer unit d = Y_max / 2^(Q+8) (256 accumulator steps per half level):
 *          E = x (2b+1) 256 + W S + Qd with W = rint(fl32(w Rd)),
 *          Qd = rint(fl32(q Rd)), Rd = fl32(2^(Q+8) / Y_max), compared with
 *          Theta(u) = rint(fl32(fl32(theta lambda^u) Rd)).  Only the held sample
 *          is quantized to Q bits; the perturbation, the weight and the
 *          threshold keep the accumulator's resolution.
 *
 * Uniform perturbation (Sec. V-B: uniform samples may replace the Gaussian
 * ones): with the UNIFORM variant bit, output r of the same Philox counter
 * gives v = (2 (r >> 8) + 1 - 2^24) 2^-24, uniform on (-1, 1) and exact in
 * FP32, and q_k = fl32(eta sigma sqrt 3) v (same variance eta^2 sigma^2 as the
 * Gaussian perturbation; the paper does not state the variance, so equal
 * variance is the reading taken).
 *
 * Objective trace (Sec. III-B, the GDBF objective f(x) = sum_k x_k y_k +
 * sum_i s_i, tracked over iterations in Sec. VI): for traced frames, at every
 * syndrome test t the decoder records U(t), the number of unsatisfied checks
 * (so sum_i s_i = m - 2 U(t)), and C(t) = sum_k rint(x_k(t) y~_k 2^32), the
 * correlation with the held samples y~ as an exact integer in units of 2^-32
 * (each term is exact in double; rint only rounds terms below 2^-32, so
 * |C(t) 2^-32 - sum_k x_k y~_k| <= n 2^-33).  f(x(t)) = C(t) 2^-32 + m - 2U(t).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_ADAPT 1
#define ORC_SMOOTH 2
#define ORC_SINGLE 4
#define ORC_UNIFORM 8
#define ORC_FP32 0
#define ORC_FP16 1
#define ORC_FIX 2
#define ORC_FIXACC 3
#define ORC_ACC_BITS 8          /* accumulator steps per half level: 2^8 */

typedef struct {
    float w, theta, eta, lambda, y_max;
    int32_t t_max, smooth_window, variant, precision, q_bits;
} orc_params;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10                                                             */
/* ------------------------------------------------------------------------ */

void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    const uint32_t mul0 = 0xD2511F53u, mul1 = 0xCD9E8D57u;   /* round multipliers */
    const uint32_t bump0 = 0x9E3779B9u, bump1 = 0xBB67AE85u; /* Weyl key increments */
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        uint64_t p0 = (uint64_t)mul0 * c0;
        uint64_t p1 = (uint64_t)mul1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += bump0; k1 += bump1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------ */
/* Standard normal deviates by inversion of the normal CDF                   */
/* ------------------------------------------------------------------------ */

/* One Philox output r gives one deviate.  Bit 31 is the sign; the other 31
 * bits give the lower-tail probability p = (2 (r mod 2^31) + 1) 2^-33, which
 * lies in (0, 1/2) and is exact in double; the deviate is -Phi^{-1}(p) when bit
 * 31 is set and Phi^{-1}(p) otherwise (the inversion method applied to the
 * symmetric uniform u = p or 1 - p).
 *
 * FP32 form: with a = 2 (r mod 2^31) + 1 and j the number of leading zeros of
 * the 32-bit a, p lies in the dyadic interval [2^-(j+2), 2^-(j+1)); the three
 * bits after the leading one of a pick one of eight equal sub-intervals
 * (segment (j, s), 32 x 8 segments), and the next 23 bits give the position
 * v in [-1/2, 1/2) inside it, so p = (8 + s + 1/2 + v) 2^-(j+5) (bits of a
 * beyond those are dropped).  On each segment Phi^{-1} is replaced by the
 * cubic in v that interpolates it at the four Chebyshev nodes
 * v_i = cos((2i+1) pi / 8) / 2, with FP32 coefficients (table below), and
 * evaluated by Horner's rule with fused multiply-adds.
 *
 * FP64 form: two Newton steps on Phi(z) = p from the FP32 value, with Phi
 * from the C library's erfc. */

/* Phi(z) = erfc(-z / sqrt 2) / 2 */
static double phi_cdf(double z) { return 0.5 * erfc(-z * 0.70710678118654752); }

/* Phi^{-1}(p) for 0 < p < 1/2 in double: 100 bisection steps of Phi(z) = p on
 * [-40, 0], which end on adjacent doubles. */
static double inv_phi_bisect(double p) {
    double lo = -40.0, hi = 0.0;
    for (int it = 0; it < 100; ++it) {
        double mid = 0.5 * (lo + hi);
        if (phi_cdf(mid) < p) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* icdf_tab[j][s] = FP32 coefficients c0..c3 of segment (j, s).  The cubic
 * through (v_i, g_i), g_i = Phi^{-1}(p(v_i)), in the Chebyshev basis
 * T_n(2v): b0 = sum g_i / 4, b_n = sum g_i T_n(x_i) / 2 (x_i = 2 v_i), with
 * T_1(x_i) = x_i, T_2(x_i) = +-sqrt(2)/2, T_3(x_i) = (C3, -C1, C1, -C3) for
 * C1 = cos(pi/8), C3 = cos(3pi/8); then T_1(2v) = 2v, T_2(2v) = 8v^2 - 1,
 * T_3(2v) = 32v^3 - 6v give c0 = b0 - b2, c1 = 2 b1 - 6 b3, c2 = 8 b2,
 * c3 = 32 b3.  All in double, in this order, then rounded to FP32. */
static float icdf_tab[32][8][4];
static pthread_once_t icdf_once = PTHREAD_ONCE_INIT;

static void icdf_init(void) {
    const double C1 = 0.5 * sqrt(2.0 + sqrt(2.0)), C3 = 0.5 * sqrt(2.0 - sqrt(2.0));
    const double R = 0.5 * sqrt(2.0);
    const double node[4] = {0.5 * C1, 0.5 * C3, -0.5 * C3, -0.5 * C1};
    for (int j = 0; j < 32; ++j)
        for (int s = 0; s < 8; ++s) {
            double g[4];
            for (int i = 0; i < 4; ++i)
                g[i] = inv_phi_bisect(ldexp(8.0 + s + 0.5 + node[i], -(j + 5)));
            double d03 = g[0] - g[3], d12 = g[1] - g[2], s03 = g[0] + g[3], s12 = g[1] + g[2];
            double b0 = (s03 + s12) * 0.25;
            double b1 = (d03 * C1 + d12 * C3) * 0.5;
            double b2 = ((s03 - s12) * R) * 0.5;
            double b3 = (d03 * C3 - d12 * C1) * 0.5;
            icdf_tab[j][s][0] = (float)(b0 - b2);
            icdf_tab[j][s][1] = (float)(2.0 * b1 - 6.0 * b3);
            icdf_tab[j][s][2] = (float)(8.0 * b2);
            icdf_tab[j][s][3] = (float)(32.0 * b3);
        }
}

void oracle_icdf_table(float* out) {
    pthread_once(&icdf_once, icdf_init);
    memcpy(out, icdf_tab, sizeof icdf_tab);
}

/* The FP32 deviate of one Philox output. */
float oracle_gauss_f32(uint32_t r) {
    pthread_once(&icdf_once, icdf_init);
    uint32_t a = ((r & 0x7FFFFFFFu) << 1) | 1u;
    int j = 0;
    while (!(a & 0x80000000u)) { a <<= 1; ++j; }       /* a is now normalized */
    int s = (int)((a >> 28) & 7u);
    uint32_t vbits = 0x3F800000u | ((a >> 5) & 0x007FFFFFu);
    float one_plus_f;
    memcpy(&one_plus_f, &vbits, 4);
    float v = one_plus_f - 1.5f;                          /* exact */
    const float* c = icdf_tab[j][s];
    float g = fmaf(fmaf(fmaf(c[3], v, c[2]), v, c[1]), v, c[0]);
    return (r & 0x80000000u) ? -g : g;
}

/* The FP64 deviate of one Philox output. */
double oracle_gauss_f64(uint32_t r) {
    double p = ((double)(r & 0x7FFFFFFFu) * 2.0 + 1.0) * 0x1.0p-33;
    double z = (double)oracle_gauss_f32(r & 0x7FFFFFFFu);
    for (int it = 0; it < 2; ++it)
        z -= (phi_cdf(z) - p) / (exp(-0.5 * z * z) * 0.39894228040143268);
    return (r & 0x80000000u) ? -z : z;
}

/* Deviates of the outputs r[0 .. n-1] (verification). */
void oracle_gauss_many_f32(const uint32_t* r, uint32_t n, float* out) {
    for (uint32_t i = 0; i < n; ++i) out[i] = oracle_gauss_f32(r[i]);
}

/* Deviates of consecutive outputs r = start .. start + count - 1 (verification). */
void oracle_gauss_range_f32(uint32_t start, uint32_t count, float* out) {
    for (uint32_t i = 0; i < count; ++i) out[i] = oracle_gauss_f32(start + i);
}

/* Four standard normals for (seed, frame, t, symbol group g): symbol 4g + i
 * takes Philox output i of counter (g, t, frame_lo, frame_hi). */
void oracle_gauss4_f32(uint64_t seed, uint64_t frame, uint32_t t, uint32_t g, float z[4]) {
    uint32_t ctr[4] = {g, t, (uint32_t)frame, (uint32_t)(frame >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f32(r[i]);
}

void oracle_gauss4_f64(uint64_t seed, uint64_t frame, uint32_t t, uint32_t g, double z[4]) {
    uint32_t ctr[4] = {g, t, (uint32_t)frame, (uint32_t)(frame >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) z[i] = oracle_gauss_f64(r[i]);
}

/* Uniform deviate of one Philox output (Sec. V-B): the top 24 bits a = r >> 8 give
 * v = (2a + 1 - 2^24) 2^-24, an odd multiple of 2^-24 in (-1, 1): exact in FP32 and in
 * double, symmetric (v(~r) = -v(r)), variance (1 - 2^-48) / 3. */
float oracle_uniform_f32(uint32_t r) {
    const int32_t odd = (int32_t)(2u * (r >> 8) + 1u) - (1 << 24);
    return ldexpf((float)odd, -24);
}

/* Four uniform deviates for symbols 4g .. 4g+3: output i of counter (g, t, frame). */
void oracle_uniform4_f32(uint64_t seed, uint64_t frame, uint32_t t, uint32_t g, float v[4]) {
    uint32_t ctr[4] = {g, t, (uint32_t)frame, (uint32_t)(frame >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t r[4];
    oracle_philox4x32_10(ctr, key, r);
    for (int i = 0; i < 4; ++i) v[i] = oracle_uniform_f32(r[i]);
}

/* Standard deviation of q_k: eta * sigma (Sec. III-C, variance eta^2 N0/2 with
 * N0/2 = sigma^2 the channel variance), formed in double, rounded to FP32. */
static float noise_scale_f32(float eta, float sigma) { return (float)((double)eta * (double)sigma); }

/* The perturbation q_k the FP32 decoder adds for (seed, frame, t, k). */
float oracle_noise_f32(uint64_t seed, uint64_t frame, uint32_t t, uint32_t k, float eta, float sigma) {
    float z[4];
    oracle_gauss4_f32(seed, frame, t, k >> 2, z);
    return noise_scale_f32(eta, sigma) * z[k & 3];
}

/* ------------------------------------------------------------------------ */
/* Thresholds and the inversion function                                     */
/* ------------------------------------------------------------------------ */

/* theta_k = theta lambda^u (Sec. V-A, Eq. 12), tabulated for u = 0..t_max:
 * p_0 = 1, p_{u+1} = p_u * lambda in double; thr[u] = fl32(theta * p_u). */
void oracle_threshold_table_f32(float theta, float lambda, int32_t t_max, float* thr) {
    double p = 1.0;
    for (int32_t u = 0; u <= t_max; ++u) {
        thr[u] = (float)((double)theta * p);
        p = p * (double)lambda;
    }
}

/* Step 2 of Sec. III-C in FP32 with a fixed order: ((x*y) + w*S) + q. */
float oracle_metric_f32(int x, float ys, int S, float w, float q) {
    float xy = x > 0 ? ys : -ys;
    float ws = w * (float)S;
    float e = xy + ws;
    return e + q;
}

float oracle_round_half(float x);

/* Step 2 in binary16: E = h(h(x y16 + h(w16 S)) + h(q)), each result rounded to binary16. */
float oracle_metric_f16(int x, float ys16, int S, float w16, float q) {
    const float q16 = oracle_round_half(q);
    const float xy = x > 0 ? ys16 : -ys16;
    const float ws = oracle_round_half(w16 * (float)S);
    const float e1 = oracle_round_half(xy + ws);
    return oracle_round_half(e1 + q16);
}

double oracle_metric_f64(int x, double ys, int S, double w, double q) {
    return (x > 0 ? ys : -ys) + w * (double)S + q;
}

/* g(v) of Sec. IV-E, Eq. 8, with the level index saturated at 2^(Q-1)-1. */
double oracle_quantize(double v, int32_t q_bits, double y_max) {
    const double nq = ldexp(1.0, q_bits);
    double k = floor(fabs(v) * nq / (2.0 * y_max));
    const double kmax = nq / 2.0 - 1.0;
    if (k > kmax) k = kmax;
    const double s = v >= 0.0 ? 1.0 : -1.0;
    return s * (k + 0.5) * (2.0 * y_max / nq);
}

/* Round a float to the nearest binary16 value (ties to even), returned as a
 * float: quantum 2^(e-10) for normal binary16 (e >= -14), 2^-24 below;
 * magnitudes >= 65520 overflow to infinity. */
float oracle_round_half(float x) {
    uint32_t b;
    memcpy(&b, &x, 4);
    const uint32_t a = b & 0x7FFFFFFFu;
    if (a >= 0x7F800000u) return x;
    if (a >= 0x477FF000u) return (b >> 31) ? -INFINITY : INFINITY;
    const int e = (int)(a >> 23) - 127;
    const double q = ldexp(1.0, e >= -14 ? e - 10 : -24);
    const double r = rint(fabs((double)x) / q) * q;     /* exact quotient, ties to even */
    return (float)((b >> 31) ? -r : r);
}

/* R = fl32(2^Q / (2 Y_max)) of the fixed-point quantizer. */
float oracle_fix_scale(int32_t q_bits, float y_max) {
    return (float)(ldexp(1.0, q_bits) / (2.0 * (double)y_max));
}

/* Signed level code b of v (value 2b + 1 in units of Delta/2); the level is
 * decided in FP32 and saturates at kmax = 2^(Q-1) - 1. */
int32_t oracle_fix_code(float v, float R, int32_t kmax) {
    const float a = fabsf(v) * R;
    const int32_t k = (a < (float)kmax) ? (int32_t)floorf(a) : kmax;
    return v >= 0.0f ? k : -k - 1;
}

static inline int32_t fix_value(float v, float R, int32_t kmax) { return 2 * oracle_fix_code(v, R, kmax) + 1; }

/* Rd = fl32(2^(Q+8) / Y_max): accumulator steps per unit of the FIXACC form. */
float oracle_fixacc_scale(int32_t q_bits, float y_max) {
    return (float)(ldexp(1.0, q_bits + ORC_ACC_BITS) / (double)y_max);
}

/* v in accumulator steps: the FP32 product v Rd rounded to the nearest integer (ties to even). */
int32_t oracle_fixacc_steps(float v, float Rd) {
    const float a = v * Rd;
    return (int32_t)lrintf(a);
}

/* Whether the FIXACC integers stay far inside int32: |theta| Rd, w Rd 64 and the largest
 * perturbation (8 scale) Rd below 2^28. */
int oracle_fixacc_in_range(float theta, float w, float scale, float Rd) {
    const double lim = ldexp(1.0, 28);
    return fabs((double)theta) * Rd < lim && (double)w * Rd * 64.0 < lim && 8.0 * (double)scale * Rd < lim;
}

/* Adaptation events (theta~, tau~) of Sec. V-A: tau where g(theta lambda^u)
 * changes, for u = 0..t_max (Table II).  Returns the event count. */
int32_t oracle_threshold_events(double theta, double lambda, int32_t t_max, int32_t q_bits,
                                double y_max, double* thr_out, int32_t* tau_out, int32_t cap) {
    int32_t count = 0;
    double prev = 0.0;
    for (int32_t u = 0; u <= t_max; ++u) {
        double th = oracle_quantize(theta * pow(lambda, (double)u), q_bits, y_max);
        if (u == 0 || th != prev) {
            if (count < cap) { thr_out[count] = th; tau_out[count] = u; }
            ++count;
            prev = th;
        }
    }
    return count;
}

/* ------------------------------------------------------------------------ */
/* Decoder                                                                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n, m;
    const int32_t* row_ptr;   /* N(i) = col_idx[row_ptr[i] .. row_ptr[i+1]) */
    const int32_t* col_idx;
    int32_t* sym_ptr;         /* M(k) = chk_idx[sym_ptr[k] .. sym_ptr[k+1]) */
    int32_t* chk_idx;
} orc_code;

static int code_init(orc_code* C, int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx) {
    C->n = n; C->m = m; C->row_ptr = row_ptr; C->col_idx = col_idx;
    int32_t nnz = row_ptr[m];
    C->sym_ptr = (int32_t*)calloc((size_t)n + 1, sizeof(int32_t));
    C->chk_idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
    if (!C->sym_ptr || !C->chk_idx) return -1;
    for (int32_t e = 0; e < nnz; ++e) C->sym_ptr[col_idx[e] + 1]++;
    for (int32_t k = 0; k < n; ++k) C->sym_ptr[k + 1] += C->sym_ptr[k];
    int32_t* fill = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!fill) return -1;
    memcpy(fill, C->sym_ptr, sizeof(int32_t) * (size_t)n);
    for (int32_t i = 0; i < m; ++i)
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; ++e) C->chk_idx[fill[col_idx[e]]++] = i;
    free(fill);
    return 0;
}

static void code_free(orc_code* C) { free(C->sym_ptr); free(C->chk_idx); }

/* Writes x (bit 1 <=> x_k = -1, LSB-first) into out[ceil(n/8)]. */
static void pack_bits(const int8_t* x, int32_t n, uint8_t* out) {
    memset(out, 0, (size_t)(n + 7) / 8);
    for (int32_t k = 0; k < n; ++k)
        if (x[k] < 0) out[k >> 3] |= (uint8_t)(1u << (k & 7));
}

typedef struct {
    const orc_code* C;
    const orc_params* P;
    int use_f64;
    float scale32;            /* fl32(eta * sigma) */
    double scale64;           /* eta * sigma */
    const float* thr32;       /* [t_max + 1] */
    const double* thr64;
    uint64_t seed;
    const float* q_in;        /* optional [t_max][n] perturbations for one frame */
    int precision;            /* ORC_FP32, ORC_FP16 or ORC_FIX */
    float w16;                /* binary16 syndrome weight */
    const float* thr16;       /* [t_max + 1] binary16 thresholds */
    float fix_R;              /* fixed-point scale and limits */
    int32_t fix_kmax, fix_W;
    const int32_t* thr_fix;   /* [t_max + 1] Theta~(u) (FIX) or Theta(u) in steps (FIXACC) */
    float acc_R;              /* FIXACC: Rd and the weight in steps */
    int32_t acc_W;
    double y_unit;            /* FIX / FIXACC: value of one half level, Y_max 2^-Q */
} orc_ctx;

/* Correlation sum_k rint(x_k y~_k 2^32) of the objective trace (exact integer). */
static int64_t trace_corr(const orc_ctx* X, const int8_t* x, const double* ys64, const int32_t* yfix, int32_t n) {
    int64_t c = 0;
    for (int32_t k = 0; k < n; ++k) {
        const double yv = (X->precision == ORC_FIX || X->precision == ORC_FIXACC) ? (double)yfix[k] * X->y_unit
                                                                                  : ys64[k];
        c += (int64_t)llrint(ldexp((double)x[k] * yv, 32));
    }
    return c;
}

/* Decodes one frame.  ws must hold 4n + m + 16 int32 words.  tr_u / tr_c (or NULL):
 * objective trace U(t), C(t) for t = 0 .. iters. */
static void decode_frame(const orc_ctx* X, const float* y, uint64_t frame_id,
                         uint8_t* bits, int32_t* iters, uint8_t* pass, int32_t* ws,
                         int32_t* tr_u, int64_t* tr_c) {
    const orc_code* C = X->C;
    const orc_params* P = X->P;
    const int32_t n = C->n, m = C->m, T = P->t_max;
    const int adapt = (P->variant & ORC_ADAPT) != 0;
    const int smooth = (P->variant & ORC_SMOOTH) != 0;
    const int single = (P->variant & ORC_SINGLE) != 0;
    const int uniform = (P->variant & ORC_UNIFORM) != 0;
    const int fixed = X->precision == ORC_FIX || X->precision == ORC_FIXACC;
    int8_t* x = (int8_t*)ws;                       /* n bytes */
    int8_t* s = (int8_t*)(ws + (n + 3) / 4);       /* m bytes */
    int32_t* u = ws + (n + 3) / 4 + (m + 3) / 4;   /* n */
    int32_t* Xs = u + n;                           /* n */
    float* ys32 = (float*)(Xs + n);                /* n */
    double* ys64 = (double*)malloc(sizeof(double) * (size_t)n);
    int32_t* yfix = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    const int clamp = P->y_max > 0.0f && isfinite(P->y_max);

    /* Step 0 and x(0) = sign(y) on saturated samples (Sec. III-A, IV-A). */
    for (int32_t k = 0; k < n; ++k) {
        float v = y[k];
        if (clamp) { if (v > P->y_max) v = P->y_max; if (v < -P->y_max) v = -P->y_max; }
        if (X->precision == ORC_FP16) v = oracle_round_half(v);
        ys32[k] = v;
        ys64[k] = (double)v;
        x[k] = v >= 0.0f ? 1 : -1;
        if (fixed) {
            yfix[k] = fix_value(v, X->fix_R, X->fix_kmax);
            x[k] = yfix[k] > 0 ? 1 : -1;
        }
        u[k] = 0;
        Xs[k] = 0;
    }
    const int32_t t_smooth = smooth ? (T - P->smooth_window > 0 ? T - P->smooth_window : 0) : T + 1;
    float z32[4] = {0, 0, 0, 0};
    double z64[4] = {0, 0, 0, 0};

    for (int32_t t = 0; t <= T; ++t) {
        /* Step 1: syndromes and the stopping test. */
        int all_satisfied = 1;
        int32_t unsat = 0;
        for (int32_t i = 0; i < m; ++i) {
            int prod = 1;
            for (int32_t e = C->row_ptr[i]; e < C->row_ptr[i + 1]; ++e) prod *= x[C->col_idx[e]];
            s[i] = (int8_t)prod;
            if (prod < 0) { all_satisfied = 0; ++unsat; }
        }
        /* objective trace: f(x(t)) = C(t) 2^-32 + m - 2 U(t) */
        if (tr_u) {
            tr_u[t] = unsat;
            tr_c[t] = trace_corr(X, x, ys64, yfix, n);
        }
        if (all_satisfied) {
            pack_bits(x, n, bits);
            *iters = t;
            *pass = 1;
            free(ys64);
            free(yfix);
            return;
        }
        /* Eq. 7: the up/down counter sums x(t) over the smoothing window. */
        if (t >= t_smooth)
            for (int32_t k = 0; k < n; ++k) Xs[k] += x[k];
        if (t == T) break;
        /* Step 2 (noisy inversion function) and Step 3b (flip / adapt), or Step 3a
         * (single-bit): find the first k with the least E_k, flip it after the sweep. */
        int32_t best_k = -1;
        double best64 = 0.0;
        float best32 = 0.0f;
        int32_t best_fix = 0;
        for (int32_t k = 0; k < n; ++k) {
            int S = 0;
            for (int32_t e = C->sym_ptr[k]; e < C->sym_ptr[k + 1]; ++e) S += s[C->chk_idx[e]];
            int flip;
            if (X->use_f64) {
                if ((k & 3) == 0) {
                    if (uniform) {
                        oracle_uniform4_f32(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z32);
                        for (int i = 0; i < 4; ++i) z64[i] = (double)z32[i];
                    } else {
                        oracle_gauss4_f64(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z64);
                    }
                }
                double q = X->scale64 * z64[k & 3];
                double E = oracle_metric_f64(x[k], ys64[k], S, (double)P->w, q);
                flip = E < X->thr64[u[k]];
                if (single && (best_k < 0 || E < best64)) { best_k = k; best64 = E; }
            } else {
                float q;
                if (X->q_in) {
                    q = X->q_in[(size_t)t * n + k];
                } else {
                    if ((k & 3) == 0) {
                        if (uniform) oracle_uniform4_f32(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z32);
                        else oracle_gauss4_f32(X->seed, frame_id, (uint32_t)t, (uint32_t)(k >> 2), z32);
                    }
                    q = X->scale32 * z32[k & 3];
                }
                if (X->precision == ORC_FP16) {
                    const float E = oracle_metric_f16(x[k], ys32[k], S, X->w16, q);
                    flip = E < X->thr16[u[k]];
                    if (single && (best_k < 0 || E < best32)) { best_k = k; best32 = E; }
                } else if (X->precision == ORC_FIX) {
                    /* Eq. 9 in units of Delta/2: exact integers */
                    const int32_t Eq = x[k] * yfix[k] + X->fix_W * S + fix_value(q, X->fix_R, X->fix_kmax);
                    flip = Eq < X->thr_fix[u[k]];
                    if (single && (best_k < 0 || Eq < best_fix)) { best_k = k; best_fix = Eq; }
                } else if (X->precision == ORC_FIXACC) {
                    /* the held Eq. 8 level in accumulator steps (2^8 per half level), the
                     * weight, the perturbation and the threshold in the same steps: exact int32 */
                    const int32_t Ea = x[k] * yfix[k] * (1 << ORC_ACC_BITS) + X->acc_W * S +
                                       oracle_fixacc_steps(q, X->acc_R);
                    flip = Ea < X->thr_fix[u[k]];
                    if (single && (best_k < 0 || Ea < best_fix)) { best_k = k; best_fix = Ea; }
                } else {
                    float E = oracle_metric_f32(x[k], ys32[k], S, P->w, q);
                    flip = E < X->thr32[u[k]];
                    if (single && (best_k < 0 || E < best32)) { best_k = k; best32 = E; }
                }
            }
            if (single) continue;
            if (flip) x[k] = (int8_t)-x[k];
            else if (adapt) u[k] += 1;
        }
        if (single) x[best_k] = (int8_t)-x[best_k];
    }
    /* T reached: smoothed decision sign(X_k) (Sec. III-E), zero keeps x_k(T). */
    if (smooth)
        for (int32_t k = 0; k < n; ++k) x[k] = Xs[k] > 0 ? 1 : (Xs[k] < 0 ? -1 : x[k]);
    pack_bits(x, n, bits);
    *iters = T;
    *pass = 0;
    free(ys64);
    free(yfix);
}

typedef struct {
    const orc_ctx* X;
    const float* y;
    int64_t f0, f1;
    uint64_t frame_offset;
    uint8_t* bits;
    int32_t* iters;
    uint8_t* pass;
    int64_t trace_frames;     /* frames 0 .. trace_frames-1 of the call are traced */
    int32_t* tr_u;            /* [trace_frames][t_max + 1] */
    int64_t* tr_c;
    int status;
} orc_job;

static void* decode_worker(void* arg) {
    orc_job* J = (orc_job*)arg;
    const orc_code* C = J->X->C;
    const int32_t n = C->n, nb = (C->n + 7) / 8;
    int32_t* ws = (int32_t*)malloc(sizeof(int32_t) * (size_t)(4 * n + C->m + 16));
    if (!ws) { J->status = -1; return NULL; }
    const int64_t tl = (int64_t)J->X->P->t_max + 1;
    for (int64_t f = J->f0; f < J->f1; ++f) {
        const int traced = f < J->trace_frames;
        decode_frame(J->X, J->y + f * (int64_t)n, J->frame_offset + (uint64_t)f,
                     J->bits + f * (int64_t)nb, J->iters + f, J->pass + f, ws,
                     traced ? J->tr_u + f * tl : NULL, traced ? J->tr_c + f * tl : NULL);
    }
    free(ws);
    J->status = 0;
    return NULL;
}

static int check_args(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                      const orc_params* P) {
    if (n <= 0 || m <= 0 || !row_ptr || !col_idx || !P) return -1;
    if (row_ptr[0] != 0) return -1;
    for (int32_t i = 0; i < m; ++i) if (row_ptr[i + 1] < row_ptr[i]) return -1;
    for (int32_t e = 0; e < row_ptr[m]; ++e) if (col_idx[e] < 0 || col_idx[e] >= n) return -1;
    if (P->t_max < 0 || P->smooth_window < 0) return -1;
    if (P->precision < ORC_FP32 || P->precision > ORC_FIXACC) return -1;
    if (P->variant & ~(ORC_ADAPT | ORC_SMOOTH | ORC_SINGLE | ORC_UNIFORM)) return -1;
    if ((P->variant & ORC_SINGLE) && (P->variant & ORC_ADAPT)) return -1;
    if ((P->precision == ORC_FIX || P->precision == ORC_FIXACC) &&
        (P->q_bits < 2 || P->q_bits > 8 || !(P->y_max > 0.0f) || !isfinite(P->y_max)))
        return -1;
    return 0;
}

static int run(int use_f64, int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
               const float* y, int64_t n_frames, float sigma, const orc_params* P, uint64_t seed,
               uint64_t frame_offset, const float* q_in, uint8_t* bits, int32_t* iters,
               uint8_t* pass, int32_t n_threads, int64_t trace_frames, int32_t* tr_u, int64_t* tr_c) {
    if (check_args(n, m, row_ptr, col_idx, P) != 0 || n_frames < 0) return -1;
    /* the trace needs bounded samples: a finite saturation level below 2^30 */
    if (trace_frames > 0 && (!tr_u || !tr_c || !(P->y_max > 0.0f) || !(P->y_max < 1073741824.0f))) return -1;
    if (n_frames == 0) return 0;
    orc_code C;
    if (code_init(&C, n, m, row_ptr, col_idx) != 0) { code_free(&C); return -1; }
    float* thr32 = (float*)malloc(sizeof(float) * (size_t)(P->t_max + 1));
    double* thr64 = (double*)malloc(sizeof(double) * (size_t)(P->t_max + 1));
    oracle_threshold_table_f32(P->theta, P->lambda, P->t_max, thr32);
    for (int32_t u = 0; u <= P->t_max; ++u) thr64[u] = (double)P->theta * pow((double)P->lambda, (double)u);
    float* thr16 = (float*)malloc(sizeof(float) * (size_t)(P->t_max + 1));
    int32_t* thr_fix = (int32_t*)malloc(sizeof(int32_t) * (size_t)(P->t_max + 1));
    orc_ctx X;
    X.precision = use_f64 ? ORC_FP32 : P->precision;
    X.w16 = oracle_round_half(P->w);
    X.fix_R = 0.0f; X.fix_kmax = 0; X.fix_W = 0;
    X.acc_R = 0.0f; X.acc_W = 0; X.y_unit = 0.0;
    if (X.precision == ORC_FIX || X.precision == ORC_FIXACC) {
        X.fix_R = oracle_fix_scale(P->q_bits, P->y_max);
        X.fix_kmax = (1 << (P->q_bits - 1)) - 1;
        X.fix_W = fix_value(P->w, X.fix_R, X.fix_kmax);
        X.y_unit = ldexp((double)P->y_max, -P->q_bits);
    }
    const int uniform = (P->variant & ORC_UNIFORM) != 0;
    /* perturbation scale: eta sigma (Gaussian) or eta sigma sqrt 3 (uniform on (-1, 1)) */
    const double scale_d = uniform ? ((double)P->eta * (double)sigma) * sqrt(3.0) : (double)P->eta * (double)sigma;
    if (X.precision == ORC_FIXACC) {
        X.acc_R = oracle_fixacc_scale(P->q_bits, P->y_max);
        X.acc_W = oracle_fixacc_steps(P->w, X.acc_R);
        if (!oracle_fixacc_in_range(P->theta, P->w, (float)scale_d, X.acc_R)) {
            free(thr32); free(thr64); free(thr16); free(thr_fix);
            code_free(&C);
            return -1;
        }
    }
    for (int32_t u = 0; u <= P->t_max; ++u) {
        thr16[u] = oracle_round_half(thr32[u]);
        thr_fix[u] = X.precision == ORC_FIX ? fix_value(thr32[u], X.fix_R, X.fix_kmax)
                   : X.precision == ORC_FIXACC ? oracle_fixacc_steps(thr32[u], X.acc_R) : 0;
    }
    X.thr16 = thr16;
    X.thr_fix = thr_fix;
    X.C = &C; X.P = P; X.use_f64 = use_f64;
    X.scale32 = (float)scale_d;
    X.scale64 = scale_d;
    X.thr32 = thr32; X.thr64 = thr64; X.seed = seed; X.q_in = q_in;
    if (n_threads <= 0) n_threads = 1;
    if (n_threads > 512) n_threads = 512;
    if (n_frames < n_threads) n_threads = (int32_t)n_frames;
    pthread_t th[512];
    orc_job jobs[512];
    for (int32_t i = 0; i < n_threads; ++i) {
        jobs[i].X = &X; jobs[i].y = y;
        jobs[i].f0 = n_frames * i / n_threads; jobs[i].f1 = n_frames * (i + 1) / n_threads;
        jobs[i].frame_offset = frame_offset;
        jobs[i].bits = bits; jobs[i].iters = iters; jobs[i].pass = pass; jobs[i].status = 0;
        jobs[i].trace_frames = trace_frames; jobs[i].tr_u = tr_u; jobs[i].tr_c = tr_c;
    }
    for (int32_t i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, decode_worker, &jobs[i]);
    decode_worker(&jobs[0]);
    int status = jobs[0].status;
    for (int32_t i = 1; i < n_threads; ++i) { pthread_join(th[i], NULL); status |= jobs[i].status; }
    free(thr32); free(thr64); free(thr16); free(thr_fix);
    code_free(&C);
    return status;
}

/* FP32 decoder with a fixed operation order: the bit-exact reference. */
int oracle_decode_f32(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                      const float* y, int64_t n_frames, float sigma, const orc_params* P,
                      uint64_t seed, uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                      uint8_t* pass, int32_t n_threads) {
    return run(0, n, m, row_ptr, col_idx, y, n_frames, sigma, P, seed, frame_offset, NULL,
               bits, iters, pass, n_threads, 0, NULL, NULL);
}

/* FP32 decoder with the objective trace of frames 0 .. trace_frames-1:
 * tr_u / tr_c [trace_frames][t_max + 1], entries t = 0 .. iters[f] written. */
int oracle_decode_f32_trace(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                            const float* y, int64_t n_frames, float sigma, const orc_params* P,
                            uint64_t seed, uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                            uint8_t* pass, int32_t n_threads, int64_t trace_frames, int32_t* tr_u,
                            int64_t* tr_c) {
    return run(0, n, m, row_ptr, col_idx, y, n_frames, sigma, P, seed, frame_offset, NULL,
               bits, iters, pass, n_threads, trace_frames, tr_u, tr_c);
}

/* FP64 decoder on the same Philox outputs: the statistical reference. */
int oracle_decode_f64(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                      const float* y, int64_t n_frames, float sigma, const orc_params* P,
                      uint64_t seed, uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                      uint8_t* pass, int32_t n_threads) {
    return run(1, n, m, row_ptr, col_idx, y, n_frames, sigma, P, seed, frame_offset, NULL,
               bits, iters, pass, n_threads, 0, NULL, NULL);
}

int oracle_decode_f64_trace(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                            const float* y, int64_t n_frames, float sigma, const orc_params* P,
                            uint64_t seed, uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                            uint8_t* pass, int32_t n_threads, int64_t trace_frames, int32_t* tr_u,
                            int64_t* tr_c) {
    return run(1, n, m, row_ptr, col_idx, y, n_frames, sigma, P, seed, frame_offset, NULL,
               bits, iters, pass, n_threads, trace_frames, tr_u, tr_c);
}

/* FP32 decoder of ONE frame with the perturbations given: q[t][k], t < t_max. */
int oracle_decode_f32_qin(int32_t n, int32_t m, const int32_t* row_ptr, const int32_t* col_idx,
                          const float* y, const orc_params* P, const float* q,
                          uint8_t* bits, int32_t* iters, uint8_t* pass) {
    return run(0, n, m, row_ptr, col_idx, y, 1, 0.0f, P, 0, 0, q, bits, iters, pass, 1, 0, NULL, NULL);
}
