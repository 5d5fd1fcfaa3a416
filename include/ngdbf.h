/*
 * ngdbf.h -- C ABI of the GB300 Noisy Gradient Descent Bit-Flip (NGDBF)
 * LDPC decoder.
 *
 * Method: Sundararajan, Winstead, Boutillon, "Noisy Gradient Descent
 * Bit-Flip Decoding for LDPC Codes", IEEE Trans. Commun. 62(10), 2014.
 *   Sec. III-A  code, channel and notation: H (m x n, n > m >= 1), bipolar
 *               codewords 1 - 2c, y = c^ + z with var(z) = N0/2,
 *               x(0) = sign(y), N(i), M(k), s_i = prod_{j in N(i)} x_j
 *   Sec. III-B  Step 1 (syndromes, stop when all s_i = +1), Step 3b
 *               (multi-bit flip when E_k < theta), Step 4 (repeat to T)
 *   Sec. III-C  Step 2: E_k = x_k y_k + w sum_{i in M(k)} s_i + q_k,
 *               q_k ~ N(0, eta^2 N0/2)
 *   Sec. III-D  threshold adaptation: theta_k <- theta_k lambda when x_k is
 *               not flipped (implemented as theta lambda^{u_k}, Sec. V-A,
 *               Eqs. 11-12, u_k = number of non-flips)
 *   Sec. III-E  output smoothing, Eq. 7: up/down counter X_k over
 *               t = T-W .. T, output sign(X_k) when T is reached
 *
 * Conventions shared by every entry point:
 *   - Bits: bit k of frame f is byte f*ceil(n/8) + k/8, bit k%8 (LSB
 *     first); bit 1 <=> x_k = -1 <=> c_k = 1.
 *   - Samples are saturated to [-y_max, y_max] first (Sec. IV-A), sign(0)
 *     is +1.  Decisions E_k < theta_k flip; a tie does not flip.
 *   - iters[f] = iteration t at which all checks were satisfied (0 for a
 *     valid input), or t_max when the limit was reached; pass[f] = 1 iff
 *     all checks were satisfied (the smoothed output is not re-checked).
 *   - q_k is drawn by Philox4x32-10 (Salmon et al., SC'11) keyed by
 *     (seed_lo, seed_hi) with counter (k/4, t, frame_lo, frame_hi), where
 *     frame = frame_offset + index of the frame in the call; symbol 4g + i
 *     takes output r_i, mapped to a standard normal deviate z by inversion
 *     of the normal CDF: bit 31 of r is the sign, p = (2 (r mod 2^31) + 1)
 *     2^-33, and Phi^{-1}(p) is evaluated in FP32 as a cubic in the position
 *     of p inside one of 32 x 8 segments (dyadic intervals of p, each split
 *     in eight), with coefficients that interpolate Phi^{-1} at the segment's
 *     Chebyshev nodes (ngdbf_gaussian_range exposes the deviates).  The
 *     perturbation is fl32(eta * sigma) * z.  A frame's result therefore
 *     depends only on (y, sigma, params, seed, frame id): never on the other
 *     frames of the call or on the launch shape.
 *   - Errors: every function returns a status and never aborts;
 *     ngdbf_last_error() gives a message for the calling thread.  CUDA
 *     errors raised by earlier asynchronous work may surface on a later call.
 */
#ifndef NGDBF_H
#define NGDBF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    NGDBF_OK = 0,
    NGDBF_ERR_INVALID_ARG = 1,   /* bad pointer, size, index or parameter */
    NGDBF_ERR_OOM = 2,           /* device or host allocation failed */
    NGDBF_ERR_CUDA = 3,          /* a CUDA runtime call failed */
    NGDBF_ERR_UNSUPPORTED = 4,   /* valid input outside this build's limits */
    NGDBF_ERR_TIMEOUT = 5        /* a wait ran out of time */
} ngdbf_status;

/* Variant bits (Sec. III-C/D/E).  0 = plain M-NGDBF with one threshold.
 * NGDBF_SINGLE: S-NGDBF, Step 3a of Sec. III-B with the noisy Step 2 of Sec. III-C:
 * each iteration flips only the symbol with the least E_k (ties go to the lowest k);
 * no threshold, so it excludes NGDBF_ADAPT; NGDBF_SMOOTH may be added.
 * NGDBF_UNIFORM: uniform instead of Gaussian perturbation samples (Sec. V-B), with the
 * same variance: output r of the same Philox counter gives v = (2 (r >> 8) + 1 - 2^24)
 * 2^-24, uniform on (-1, 1), and q_k = fl32(eta sigma sqrt 3) v.  Combines with any of
 * the other bits. */
enum { NGDBF_ADAPT = 1, NGDBF_SMOOTH = 2, NGDBF_SINGLE = 4, NGDBF_UNIFORM = 8 };

/* Arithmetic of the held samples and the inversion function (Sec. IV-E); the
 * perturbation is always the FP32 generator output.
 *   NGDBF_FP32  E = ((x y + w S) + q), every step rounded to FP32.
 *   NGDBF_FP16  y, w, q and theta lambda^u rounded to binary16 (nearest even);
 *               E = h(h(x y + h(w S)) + q) with every result rounded to binary16.
 *   NGDBF_FIX   Eq. 8 with q_bits = Q (2..8): level k = min(floor(|v| R),
 *               2^(Q-1) - 1), R = fl32(2^Q / (2 y_max)), the product in FP32;
 *               value 2b + 1 (b = k, or -k-1 for v < 0) in units of y_max / 2^Q;
 *               E~ = x Y~ + W~ S + Q~ in exact integers against the level of
 *               fl32(theta lambda^u).  Samples are held in 8 bits.
 *   NGDBF_FIXACC samples held as the Eq. 8 level code of NGDBF_FIX (q_bits = Q, 8 bits
 *               each), but only the sample is quantized to Q bits: E is accumulated in
 *               exact int32 in steps of Y_max 2^-(Q+8) (256 steps per half level):
 *               E = x (2b+1) 256 + W S + rint(fl32(q Rd)), W = rint(fl32(w Rd)),
 *               Rd = fl32(2^(Q+8) / Y_max), flip when E < rint(fl32(fl32(theta
 *               lambda^u) Rd)).  The accumulator terms must stay below 2^28 steps
 *               (|theta|, 64 w and 8 eta sigma), else NGDBF_ERR_UNSUPPORTED. */
enum { NGDBF_FP32 = 0, NGDBF_FP16 = 1, NGDBF_FIX = 2, NGDBF_FIXACC = 3 };

/* Limits of this build. */
enum {
    NGDBF_MAX_T = 511,            /* t_max */
    NGDBF_MAX_WINDOW = 126,       /* smooth_window */
    NGDBF_MAX_N = 65535,          /* symbols */
    NGDBF_MAX_DEGREE = 64,        /* symbol and check degree */
    NGDBF_NOALLOC_SCRATCH_BYTES = 40 << 20   /* static scratch of ngdbf_decode_noalloc */
};

typedef struct ngdbf_params {
    float w;              /* syndrome weight w > 0 (Sec. III-C) */
    float theta;          /* initial inversion threshold (Sec. III-B), finite */
    float eta;            /* noise scale, 0 <= eta <= 1; 0 gives plain GDBF (Sec. III-C) */
    float lambda;         /* adaptation factor, 0 < lambda <= 1 (Sec. III-D) */
    float y_max;          /* saturation magnitude; <= 0 or +inf disables (Sec. IV-A) */
    int32_t t_max;        /* T: at most T flip phases, 0 <= T <= NGDBF_MAX_T */
    int32_t smooth_window;/* W: X_k sums x(t) for t = max(0, T-W) .. T, 0 <= W <= 126 */
    int32_t variant;      /* OR of NGDBF_ADAPT, NGDBF_SMOOTH, NGDBF_SINGLE (not with ADAPT), NGDBF_UNIFORM */
    int32_t precision;    /* NGDBF_FP32, NGDBF_FP16, NGDBF_FIX or NGDBF_FIXACC */
    int32_t q_bits;       /* NGDBF_FIX / NGDBF_FIXACC: Q in 2..8 (needs a finite y_max > 0); otherwise 0 */
} ngdbf_params;

typedef struct ngdbf_code ngdbf_code_t;   /* opaque; owned by the library */

/*
 * Builds the device-resident tables of a parity-check matrix H (Sec. III-A).
 *   n, m      symbols and checks, n > m >= 1, n <= NGDBF_MAX_N
 *   row_ptr   HOST int32[m+1], row_ptr[0] = 0, non-decreasing
 *   col_idx   HOST int32[row_ptr[m]]: N(i) = col_idx[row_ptr[i] .. row_ptr[i+1])
 * Every check must have degree >= 1 and every symbol degree >= 1; degrees
 * are at most NGDBF_MAX_DEGREE; no column may repeat within a row.
 * The arrays are copied; the caller keeps ownership.  On success *out
 * receives a handle that must be released with ngdbf_code_destroy.  The
 * tables live on the device that is current at this call.
 * Errors: INVALID_ARG (bad structure), UNSUPPORTED (limits), OOM, CUDA.
 */
ngdbf_status ngdbf_code_create(int32_t n, int32_t m, const int32_t* row_ptr,
                               const int32_t* col_idx, ngdbf_code_t** out);

/* Releases a code handle (NULL is accepted).  The caller must ensure no
 * decode using it is still running on the device. */
ngdbf_status ngdbf_code_destroy(ngdbf_code_t* code);

/* Reports n, m, maximum symbol degree and maximum check degree. */
ngdbf_status ngdbf_code_info(const ngdbf_code_t* code, int32_t* n, int32_t* m,
                             int32_t* dv_max, int32_t* dc_max);

/*
 * Decodes a batch of frames on the GPU (Steps 0-4 of Sec. III-B with Step 2
 * of Sec. III-C, adaptation of Sec. III-D and smoothing of Sec. III-E as
 * selected by params->variant).
 *   y            DEVICE float[n_frames][n], frame-major channel samples
 *   n_frames     >= 0 (0 returns immediately)
 *   sigma        channel noise standard deviation (N0/2 = sigma^2), >= 0
 *   seed         Philox key of the perturbation
 *   frame_offset frame id of y[0] for the perturbation counter
 *   bits         DEVICE uint8[n_frames][ceil(n/8)] decoded words (written)
 *   iters        DEVICE int32[n_frames] (written)
 *   pass         DEVICE uint8[n_frames] (written)
 *   stream       cudaStream_t to run on (NULL = legacy default stream)
 * Asynchronous: returns after enqueueing; outputs are valid once the stream
 * reaches this point.  Temporary device memory (per-slot sample copies and
 * a work counter, about 160 * n bytes per 32 concurrently decoded frames)
 * is taken from a library-owned stream-ordered pool and returned on the
 * same stream.  All pointers must be device memory of the current device.
 * The decision, syndrome and count words of one CTA's 32 frames must fit the
 * device's shared memory per block (about 20 n + 16 m + 5 KB bytes for symbol
 * degrees up to 7: n up to about 8,000 at rate 1/2 on a 227 KB device); larger
 * codes are rejected with NGDBF_ERR_UNSUPPORTED.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 */
ngdbf_status ngdbf_decode(const ngdbf_code_t* code, const float* y, int64_t n_frames,
                          float sigma, const ngdbf_params* params, uint64_t seed,
                          uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                          uint8_t* pass, void* stream);

/*
 * ngdbf_decode with the objective trace of Sec. III-B, f(x) = sum_k x_k y_k + sum_i s_i
 * (the quantity Sec. VI follows over iterations): for frames 0 .. trace_frames-1 of the
 * call, at every syndrome test t = 0 .. iters[f] the decoder records
 *   trace_unsat[f][t] = U(t), the number of unsatisfied checks of x(t), and
 *   trace_corr[f][t]  = C(t) = sum_k rint(x_k(t) y~_k 2^32), with y~ the held (saturated,
 *                       rounded or quantized) sample as an exact double,
 * so f(x(t)) = C(t) 2^-32 + m - 2 U(t) (|C 2^-32 - sum x y~| <= n 2^-33; the integer sum
 * does not depend on the order of its terms).  Entries after iters[f] are not written.
 *   trace_unsat  DEVICE int32[trace_frames][t_max + 1]
 *   trace_corr   DEVICE int64[trace_frames][t_max + 1]
 * 0 <= trace_frames <= n_frames; tracing needs a finite y_max > 0 below 2^30.  The decode
 * results equal ngdbf_decode's.  Errors: as ngdbf_decode, INVALID_ARG for bad trace buffers.
 */
ngdbf_status ngdbf_decode_trace(const ngdbf_code_t* code, const float* y, int64_t n_frames,
                                float sigma, const ngdbf_params* params, uint64_t seed,
                                uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                                uint8_t* pass, int64_t trace_frames, int32_t* trace_unsat,
                                int64_t* trace_corr, void* stream);

/*
 * The plain per-iteration form of the same decode (the baseline the persistent kernels are
 * measured against): per iteration t one launch forms the syndromes of every active frame
 * (Step 1, one thread per frame and check, one byte per decision), one retires the frames
 * that satisfy every check or reached T (outputs as ngdbf_decode's), and one runs Step 2 and
 * Step 3b for every symbol of the active frames (one thread per frame and four symbols) --
 * 3 T + 3 launches with the initializing one, no bit-slicing, no persistent slots.  Same
 * arguments, layouts and results as ngdbf_decode (bit for bit).  FP32 and the multi-bit variants only (NGDBF_SINGLE
 * and other precisions: NGDBF_ERR_UNSUPPORTED).  Scratch (about 6 n + m bytes per frame)
 * comes from the library's pool.
 */
ngdbf_status ngdbf_decode_plain(const ngdbf_code_t* code, const float* y, int64_t n_frames,
                                float sigma, const ngdbf_params* params, uint64_t seed,
                                uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                                uint8_t* pass, void* stream);

/*
 * Same decode with HOST buffers, synchronous: copies y to the device in
 * chunks on two streams, decodes each chunk as soon as it has arrived while
 * the next chunk is copied, copies the outputs back, and returns when the
 * host outputs are written.  Samples go through the library's staging buffers
 * (ngdbf_set_host_copy_mode), so any host buffer copies at full rate; with
 * direct copies, page-locked buffers overlap and pageable ones serialize.
 * Outputs are copied straight into the caller's buffers.  Same layouts as
 * ngdbf_decode.
 * chunk_frames <= 0 picks chunk sizes automatically: a quarter of the call
 * (between 256 MB and 2 GB of samples, at least 4096 frames), reached by doubling
 * from an eighth of it so that little copying precedes the first decode; two
 * chunks of device scratch are held at a time.
 */
ngdbf_status ngdbf_decode_host(const ngdbf_code_t* code, const float* y_host, int64_t n_frames,
                               float sigma, const ngdbf_params* params, uint64_t seed,
                               uint64_t frame_offset, uint8_t* bits_host, int32_t* iters_host,
                               uint8_t* pass_host, int64_t chunk_frames);

/*
 * How ngdbf_decode_host moves samples to the device (process-wide):
 * NGDBF_HOST_COPY_STAGED (default): host threads (up to 16) copy each piece of up to 128 MB
 * into one of two page-locked staging buffers that the library keeps and reuses, and the
 * device copies from there; works at the host's memcpy rate (about 120 GB/s on a 16-core
 * Grace host) whether the caller's buffer is page-locked or not, and whatever its pages.
 * NGDBF_HOST_COPY_DIRECT: the device copies straight from the caller's buffer (no host
 * threads; about 210 GB/s from page-locked memory whose translations are cheap, but on the
 * GB300 hosts measured first copies from the first several GB of page-locked memory a
 * process registered ran at 2-20 GB/s).
 * Errors: INVALID_ARG (unknown mode, NULL out).
 */
enum { NGDBF_HOST_COPY_STAGED = 0, NGDBF_HOST_COPY_DIRECT = 1 };
ngdbf_status ngdbf_set_host_copy_mode(int32_t mode);
ngdbf_status ngdbf_get_host_copy_mode(int32_t* mode);

/* Timing of the most recent ngdbf_decode_host on the calling thread, from CUDA events
 * recorded around each chunk's copy in, decode and copy out (device clock, ms): summed
 * durations of each kind, and the wall time from the first copy in to the last copy out.
 * h2d_bytes / h2d_ms is the achieved host-to-device rate; when copies overlap decoding,
 * wall_ms < h2d_ms + kernel_ms + d2h_ms.  All zero after a failed call. */
typedef struct ngdbf_host_stats {
    int32_t chunks;
    int32_t reserved;
    int64_t h2d_bytes;       /* samples copied in */
    int64_t d2h_bytes;       /* bits, iteration counts and pass flags copied out */
    double h2d_ms;
    double kernel_ms;
    double d2h_ms;
    double wall_ms;
} ngdbf_host_stats;

ngdbf_status ngdbf_last_host_stats(ngdbf_host_stats* out);

/*
 * ngdbf_decode_noalloc -- ngdbf_decode that allocates no device memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate while they decode, for example a receiver with a fixed
 * memory plan that forbids allocation after start-up (cudaMalloc may
 * synchronize the device and its latency is unbounded), or a host
 * application whose own allocator already owns the device memory.
 *
 * Same arguments, layouts and results as ngdbf_decode; the caller still
 * provides y, bits, iters and pass as device memory.  Instead of taking
 * scratch from a pool, the call uses one static device array of
 * NGDBF_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds
 * until the process exits.  Consequences:
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - Every call shares the array and its work counter (the call clears the
 *     counter on its stream before the kernel).  Calls that overlap on the
 *     GPU race and give wrong results: serialize them, e.g. on one stream.
 *   - When the per-CTA scratch of a full launch does not fit, the launch
 *     uses fewer CTAs (slower, same results); a code whose single CTA needs
 *     more than the array holds is rejected with NGDBF_ERR_UNSUPPORTED.
 * Calls no cudaMalloc, cudaFree or allocating library routine.
 */
ngdbf_status ngdbf_decode_noalloc(const ngdbf_code_t* code, const float* y, int64_t n_frames,
                                  float sigma, const ngdbf_params* params, uint64_t seed,
                                  uint64_t frame_offset, uint8_t* bits, int32_t* iters,
                                  uint8_t* pass, void* stream);

/*
 * Device memory held by the library's stream-ordered scratch pool of the current device (the
 * pool ngdbf_decode, ngdbf_decode_host and ngdbf_decode_trace take scratch from): bytes in use
 * now and the most in use since the mark was last reset; reset_high != 0 first resets the mark
 * to the current use.  Both are 0 while no decode on this device has created the pool.  Lets a
 * caller confirm that a code path (ngdbf_decode_noalloc) takes nothing from the pool.
 * Errors: INVALID_ARG for NULL outputs, CUDA.
 */
ngdbf_status ngdbf_pool_usage(int32_t reset_high, int64_t* used_now, int64_t* used_high);

/*
 * Page-locked host memory for the host-buffer entry points (ngdbf_decode_host, the server).
 * Requests of at least one transparent huge page (ngdbf_host_huge_page_bytes: 512 MiB with
 * 64 KiB base pages, 2 MiB with 4 KiB ones) are mapped on huge-page boundaries, advised for
 * huge pages (fewer translations for the copy engines) and registered with CUDA as one range
 * (the mapping rounded up to whole huge pages); smaller requests, and systems where that
 * fails, get cudaHostAlloc memory.  Contents are undefined.  The caller owns the block and
 * returns it with ngdbf_host_free (NULL: no-op).
 * Errors: INVALID_ARG (NULL out, bytes == 0, a pointer not from ngdbf_host_alloc), OOM, CUDA.
 */
ngdbf_status ngdbf_host_alloc(size_t bytes, void** out);
ngdbf_status ngdbf_host_free(void* p);
/* Transparent huge-page size the allocator aligns to (0 when the system reports none). */
ngdbf_status ngdbf_host_huge_page_bytes(int64_t* out);
/* A block from ngdbf_host_alloc: *bytes = its mapped length (0 for a cudaHostAlloc block) and
 * *huge_bytes = how much of it the kernel backs with huge pages (from /proc/self/smaps; -1 when
 * that cannot be read; huge pages are requested, not guaranteed). */
ngdbf_status ngdbf_host_block_info(const void* p, int64_t* bytes, int64_t* huge_bytes);

/*
 * Job tables: several decode jobs -- codes of different length, rate, degree
 * and iteration limit, each with its own frames, sigma and parameters -- in
 * ONE persistent launch.  CTAs start on jobs in proportion to their estimated
 * work (frames x n x (T + 1)); a CTA whose job has no unclaimed frame left and
 * whose slots are idle moves to the job with the most unclaimed work.  Each
 * frame's result is the one ngdbf_decode gives for the same job (same seed,
 * frame id = frame_offset + index): bit for bit, alone or in any mix.
 * Restrictions within one table: every job has the same params.variant and
 * params.precision; the perturbation seed is shared.
 */
typedef struct ngdbf_job {
    const ngdbf_code_t* code;
    const float* y;              /* DEVICE float[n_frames][n] */
    int64_t n_frames;
    float sigma;
    ngdbf_params params;
    uint64_t frame_offset;
    uint8_t* bits;               /* DEVICE uint8[n_frames][ceil(n/8)] */
    int32_t* iters;              /* DEVICE int32[n_frames] */
    uint8_t* pass;               /* DEVICE uint8[n_frames] */
} ngdbf_job;

typedef struct ngdbf_batch ngdbf_batch_t;   /* opaque; owns device scratch and the job table */

enum {
    NGDBF_BATCH_TUNE = 1,   /* time the candidate launch shapes on this table -- block size x
                               thread-block cluster size (1, 2, 4, 8) x split threshold (codes of
                               at least 2048, or 1024 or 4096, symbols split over the CTAs of a
                               cluster) x adjacency tables in shared memory -- and keep the fastest */
    NGDBF_BATCH_GRAPH = 2   /* capture the launch (queue reset + kernel) in a CUDA graph */
};

/*
 * Builds a launch plan for n_jobs jobs (HOST array, copied): validates every
 * job as ngdbf_decode would, uploads the job table and thresholds, allocates
 * scratch, chooses the launch shape (timed on `stream` with NGDBF_BATCH_TUNE,
 * which runs the table several times and so writes the outputs), and, with
 * NGDBF_BATCH_GRAPH, captures the launch in a CUDA graph.  The buffers named
 * by the jobs must stay valid while the batch exists.
 * Errors: INVALID_ARG, UNSUPPORTED (mixed variant or precision, limits), OOM, CUDA.
 */
ngdbf_status ngdbf_batch_create(const ngdbf_job* jobs, int32_t n_jobs, uint64_t seed, int32_t flags,
                                void* stream, ngdbf_batch_t** out);

/* Decodes every job of the table once on `stream` (asynchronous). */
ngdbf_status ngdbf_batch_launch(ngdbf_batch_t* batch, void* stream);

/* Releases the plan; no launch of it may still be running. */
ngdbf_status ngdbf_batch_destroy(ngdbf_batch_t* batch);

/*
 * Serving loop (continuous batching).  A server owns a scheduler thread, copy streams, a
 * device-memory budget and one resident persistent kernel.  Requests -- a code, HOST samples,
 * sigma, params, a frame offset and HOST output buffers -- may be submitted at any time from
 * any thread.  In arrival order, while the device memory they need (samples, outputs,
 * thresholds, and the resident kernel's scratch) fits the budget, the scheduler copies a
 * request in and publishes it into a ring of job descriptors the GPU reads.  The resident
 * kernel's CTAs take the oldest published request with frames left whenever their own is
 * exhausted, so requests that arrive while others run join the running launch and their work
 * overlaps on the device; inside a request, converged frames free their slots at once.  While
 * 16 or more published requests have frames left, a CTA whose request runs out of frames fills
 * its free slots with frames of other requests of the same code and params (chaining).  When
 * a request's last frame is done its outputs are copied back and its memory returns to the
 * budget.  When a CTA has found no work for about 20 ms the whole kernel retires (no CTA takes
 * new frames; every CTA leaves); it is launched again when work is published.  The kernel's
 * shared memory is sized for the largest code of the mix; each request is decoded in a layout
 * of its own code within it, with its per-slot state in shared memory whenever that fits
 * (requests of a code whose state does not fit use global scratch).  A request of another
 * variant or precision, or whose code needs a larger shared-memory layout, than the running
 * kernel waits until that kernel drains.  Each
 * request's result equals ngdbf_decode's for the same job, alone or in any mix; the seed of
 * the perturbation is the server's.  Samples are copied in through the library's staging
 * buffers (ngdbf_set_host_copy_mode), so any host buffer serves; with direct copies,
 * page-locked buffers let the copies run asynchronously and with pageable ones the scheduler
 * thread blocks on each copy.  Outputs are copied straight into the caller's buffers.
 */
typedef struct ngdbf_server ngdbf_server_t;

typedef struct ngdbf_server_stats {
    int64_t submitted, completed, failed;
    int64_t launches;                 /* launches of the resident kernel */
    int64_t frames;                   /* frames of completed requests */
    int64_t peak_bytes_in_use;        /* most device memory held at once (requests + kernel scratch) */
    int32_t peak_requests_on_device;  /* most requests published and not yet complete at once */
    int32_t admitted_into_running;    /* requests published while the kernel was already running */
} ngdbf_server_stats;

/* device_budget_bytes: device memory the server may hold; max_inflight_launches: 1..16 copy
 * streams; max_jobs_per_launch: 1..4096, the most requests on the device at once (at most
 * 1024 are used). */
ngdbf_status ngdbf_server_create(size_t device_budget_bytes, int32_t max_inflight_launches,
                                 int32_t max_jobs_per_launch, uint64_t seed, ngdbf_server_t** out);

/* Queues one request (validated now; HOST buffers must stay valid until the
 * request completes).  *request_id receives its id (1, 2, ...). */
ngdbf_status ngdbf_server_submit(ngdbf_server_t* server, const ngdbf_code_t* code, const float* y_host,
                                 int64_t n_frames, float sigma, const ngdbf_params* params,
                                 uint64_t frame_offset, uint8_t* bits_host, int32_t* iters_host,
                                 uint8_t* pass_host, uint64_t* request_id);

/* Completed requests not reported before, up to `capacity`: ids[i], the time
 * from submission to outputs written (seconds) and the request's status
 * (NGDBF_OK, or why it failed, e.g. NGDBF_ERR_OOM when it alone exceeds the
 * budget).  *n_out receives the count. */
ngdbf_status ngdbf_server_poll(ngdbf_server_t* server, uint64_t* ids, double* latency_s, int32_t* status,
                               int32_t capacity, int32_t* n_out);

/* Blocks until every submitted request has completed; NGDBF_ERR_TIMEOUT after timeout_s. */
ngdbf_status ngdbf_server_wait(ngdbf_server_t* server, double timeout_s);

ngdbf_status ngdbf_server_get_stats(ngdbf_server_t* server, ngdbf_server_stats* out);

/* Finishes the requests already admitted, drops the pending ones, releases everything. */
ngdbf_status ngdbf_server_destroy(ngdbf_server_t* server);

/*
 * Verification of the perturbation generator: z[i] = the standard normal deviate that
 * Philox output r = start + i (mod 2^32) gives, exactly as the decode kernels compute
 * it (inverse normal CDF, Sec. III-C draws q_k ~ N(0, eta^2 sigma^2); q_k = fl32(eta
 * sigma) * z).  Sweeping r over all 2^32 values and comparing with an independent
 * evaluation covers every deviate the generator can produce.  The paper has no
 * counterpart: its hardware draws from one shared Gaussian source (Sec. V-B).
 * z: DEVICE float[count]; asynchronous on `stream`; count = 0 is a no-op.
 * INVALID_ARG for a NULL or host z.
 */
ngdbf_status ngdbf_gaussian_range(uint32_t start, uint32_t count, float* z, void* stream);

/*
 * The perturbation generator's coefficient table (verification; host only, no device call):
 * out[4 (8 j + s) + n] = c_n of segment (j, s), the FP32 cubic in the position v of p inside
 * the segment that interpolates Phi^{-1} at the Chebyshev points (the table the kernels
 * evaluate; see the conventions at the top).  out: HOST float[1024].
 */
ngdbf_status ngdbf_generator_table(float* out);

/*
 * Same-mix throughput probe (measurement; the paper has no counterpart): every thread of a
 * full-occupancy grid runs `groups` steps of the decode's per-slot symbol work for four
 * symbols on register-resident data -- one Philox4x32-10 call, four inverse-CDF deviates
 * (coefficient table in shared memory), the FP32 inversion function from a 4-bit count lane,
 * the threshold lookup in shared memory and the comparison, the adaptation and window
 * counters, and a warp ballot rebuilding the decision word -- without the sample, state and
 * count traffic of a decode.  Timed with CUDA events, threads * groups * 4 symbols per
 * launch give the attainable rate of that instruction mix on the device.
 *   groups       >= 1 steps of four symbols per thread
 *   sink         DEVICE uint32[1], receives an XOR of every thread's result
 *   threads_out  receives the number of threads launched
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA.
 */
ngdbf_status ngdbf_mix_probe(int32_t groups, uint32_t* sink, int64_t* threads_out, void* stream);

/* Launch shape of the most recent ngdbf_decode* or ngdbf_batch_* call on the calling thread. */
typedef struct ngdbf_launch_info {
    int32_t grid;            /* CTAs (each owns 32 frame slots) */
    int32_t block;           /* threads per CTA */
    int32_t smem_bytes;      /* dynamic shared memory per CTA */
    int32_t state_in_smem;   /* 1 if per-(symbol, slot) counters live in shared memory */
    int32_t kernels;         /* kernels launched by the call */
    int32_t sm_count;        /* SMs of the device */
    int32_t tables_in_smem;  /* adjacency tables copied to shared memory: 1 N(i), 2 M(k), 3 both */
    int32_t cluster;         /* CTAs per thread-block cluster (1: none) */
    int32_t split_min_n;     /* with a cluster: codes of at least this many symbols are split over
                                it, smaller ones decoded CTA by CTA (0 without a cluster) */
} ngdbf_launch_info;

ngdbf_status ngdbf_last_launch(ngdbf_launch_info* out);

/* The candidate launch shapes of a batch, the ones NGDBF_BATCH_TUNE times (block size x
 * cluster size x split threshold x adjacency tables in shared memory; candidate 0 is the
 * default).  *count
 * (may be NULL) receives their number; info (may be NULL) receives candidate k (k < 0: the
 * shape in use): grid = the most CTAs resident at once, block, shared memory, placements
 * and cluster size. */
ngdbf_status ngdbf_batch_shape(const ngdbf_batch_t* batch, int32_t k, int32_t* count, ngdbf_launch_info* info);

/* Makes candidate k the shape of later launches (recaptures the graph of NGDBF_BATCH_GRAPH).
 * Results do not depend on the shape. */
ngdbf_status ngdbf_batch_use_shape(ngdbf_batch_t* batch, int32_t k);

/* Message for the last error on the calling thread ("" if none). */
const char* ngdbf_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* NGDBF_H */
