/*
 * Seeded synthetic workload for LDPC decoding experiments.
 *
 * This module produces the inputs that both the decoder library and the
 * reference (oracle) decoder consume.  It holds none of the decoder's
 * arithmetic: it builds a parity-check matrix, encodes random information
 * words and passes them through a binary-input AWGN channel.
 *
 *   - Parity-check matrix: progressive edge growth (Hu, Eleftheriou and
 *     Arnold, "Regular and irregular progressive edge-growth Tanner graphs",
 *     IEEE Trans. IT 51(1), 2005) with a fixed symbol degree d_v and check
 *     degrees balanced to floor/ceil of N*d_v/M.  This stands in for the
 *     MacKay codes of the paper's Sec. IV (PEGReg504x1008 and friends).
 *   - Encoding: the caller supplies, per pivot row of a reduced row-echelon
 *     form of H, a bit mask over the information positions (see the Python
 *     wrapper); parity bits are mask-and-popcount of the information word.
 *   - Channel: bipolar mapping c -> 1 - 2c (paper Sec. III-A) plus
 *     Gaussian noise of standard deviation sigma, rounded to FP32.
 *
 * Randomness comes from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014)
 * applied to (seed, domain, frame, index), so every frame is generated
 * independently of thread count and of the other frames.  Domain 1 draws
 * the information bits, domain 2 the channel noise, domain 3 the PEG ties.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t sm64_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

/* One 64-bit draw for (seed, domain, frame, index). */
static inline uint64_t wl_draw(uint64_t seed, uint64_t domain, uint64_t frame, uint64_t index) {
    uint64_t h = sm64_mix(seed ^ (domain << 56));
    h = sm64_mix(h ^ frame);
    return sm64_mix(h + index * 0xD1B54A32D192ED03ull);
}

/* ------------------------------------------------------------------------ */
/* Progressive edge growth                                                   */
/* ------------------------------------------------------------------------ */

/* Number of (check pair of v, other symbol) combinations closing a 4-cycle through v. */
static int64_t cycles4_at(int32_t v, int32_t dv, const int32_t* sadj, const int32_t* coff,
                          const int32_t* cdeg, const int32_t* cadj, int32_t* mark, int32_t* stamp) {
    int64_t cnt = 0;
    for (int32_t a = 0; a < dv; ++a) {
        int32_t ca = sadj[(int64_t)v * dv + a];
        ++*stamp;
        for (int32_t b = coff[ca]; b < coff[ca] + cdeg[ca]; ++b) mark[cadj[b]] = *stamp;
        for (int32_t a2 = a + 1; a2 < dv; ++a2) {
            int32_t cb = sadj[(int64_t)v * dv + a2];
            for (int32_t b = coff[cb]; b < coff[cb] + cdeg[cb]; ++b) {
                int32_t w = cadj[b];
                if (w != v && mark[w] == *stamp) ++cnt;
            }
        }
    }
    return cnt;
}

static void swap_slot(int32_t* arr, int32_t lo, int32_t hi, int32_t from, int32_t to) {
    for (int32_t b = lo; b < hi; ++b) if (arr[b] == from) { arr[b] = to; return; }
}

/* Degree-preserving edge swaps (v,ca),(w,cb) -> (v,cb),(w,ca) that remove the
 * 4-cycles progressive edge growth could not avoid when check capacity ran
 * out; a swap is kept only if it lowers the 4-cycle count at v and w. */
static void remove_4cycles(int32_t n, int32_t m, int32_t dv, uint64_t seed, int32_t* sadj,
                           const int32_t* coff, const int32_t* cdeg, int32_t* cadj) {
    int32_t* mark = (int32_t*)calloc((size_t)n, sizeof(int32_t));
    if (!mark) return;
    int32_t stamp = 0;
    uint64_t ctr = 0;
    const int64_t E = (int64_t)n * dv;
    for (int pass = 0; pass < 50; ++pass) {
        int changed = 0, any = 0;
        for (int32_t v = 0; v < n; ++v) {
            int64_t cv = cycles4_at(v, dv, sadj, coff, cdeg, cadj, mark, &stamp);
            if (cv == 0) continue;
            any = 1;
            for (int attempt = 0; attempt < 4000 && cv > 0; ++attempt) {
                int32_t slot_v = (int32_t)(wl_draw(seed, 3, 0xFFFFFFF0ull, ctr++) % (uint64_t)dv);
                int64_t ew = (int64_t)(wl_draw(seed, 3, 0xFFFFFFF1ull, ctr++) % (uint64_t)E);
                int32_t w = (int32_t)(ew / dv), slot_w = (int32_t)(ew % dv);
                int32_t ca = sadj[(int64_t)v * dv + slot_v], cb = sadj[(int64_t)w * dv + slot_w];
                if (w == v || ca == cb) continue;
                int clash = 0;
                for (int32_t b = 0; b < dv; ++b) {
                    clash |= sadj[(int64_t)v * dv + b] == cb;
                    clash |= sadj[(int64_t)w * dv + b] == ca;
                }
                if (clash) continue;
                int64_t before = cv + cycles4_at(w, dv, sadj, coff, cdeg, cadj, mark, &stamp);
                sadj[(int64_t)v * dv + slot_v] = cb; sadj[(int64_t)w * dv + slot_w] = ca;
                swap_slot(cadj, coff[ca], coff[ca] + cdeg[ca], v, w);
                swap_slot(cadj, coff[cb], coff[cb] + cdeg[cb], w, v);
                int64_t nv = cycles4_at(v, dv, sadj, coff, cdeg, cadj, mark, &stamp);
                int64_t after = nv + cycles4_at(w, dv, sadj, coff, cdeg, cadj, mark, &stamp);
                if (after < before) { cv = nv; changed = 1; continue; }
                sadj[(int64_t)v * dv + slot_v] = ca; sadj[(int64_t)w * dv + slot_w] = cb;
                swap_slot(cadj, coff[ca], coff[ca] + cdeg[ca], w, v);
                swap_slot(cadj, coff[cb], coff[cb] + cdeg[cb], v, w);
            }
        }
        if (!any || !changed) break;
    }
    (void)m;
    free(mark);
}

/*
 * Builds an M x N parity-check matrix with every symbol of degree dv.
 * Check i may take at most cap[i] edges, cap = floor/ceil(N*dv/M).
 * Output CSR (row_ptr[M+1], col_idx[N*dv]) with columns sorted in each row.
 * Returns 0 on success, -1 on bad arguments, -2 if some symbol could not
 * get dv distinct checks, -3 on allocation failure.
 */
int wl_peg(int32_t n, int32_t m, int32_t dv, uint64_t seed, int32_t* row_ptr, int32_t* col_idx) {
    if (n <= 0 || m <= 0 || dv <= 0 || dv > m) return -1;
    const int64_t E = (int64_t)n * dv;
    int32_t* cap = (int32_t*)malloc(sizeof(int32_t) * m);
    int32_t* cdeg = (int32_t*)calloc(m, sizeof(int32_t));
    int32_t* coff = (int32_t*)malloc(sizeof(int32_t) * (m + 1));
    int32_t* cadj = (int32_t*)malloc(sizeof(int32_t) * E);   /* check -> symbols, cap[i] slots */
    int32_t* sadj = (int32_t*)malloc(sizeof(int32_t) * E);   /* symbol -> checks, dv slots */
    int32_t* sdeg = (int32_t*)calloc(n, sizeof(int32_t));
    int32_t* cmark = (int32_t*)malloc(sizeof(int32_t) * m);  /* BFS stamp per check */
    int32_t* smark = (int32_t*)malloc(sizeof(int32_t) * n);  /* BFS stamp per symbol */
    int32_t* sq = (int32_t*)malloc(sizeof(int32_t) * n);     /* symbol frontier */
    int32_t* sq2 = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* cq = (int32_t*)malloc(sizeof(int32_t) * m);     /* checks added at the current depth */
    int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * m);
    int32_t* cdepth = (int32_t*)malloc(sizeof(int32_t) * m); /* BFS depth per check */
    int status = 0;
    if (!cap || !cdeg || !coff || !cadj || !sadj || !sdeg || !cmark || !smark || !sq || !sq2 || !cq || !cand || !cdepth) {
        status = -3;
        goto done;
    }
    {
        const int64_t base = E / m, rem = E % m;
        /* a seeded shuffle picks the `rem` checks that take one extra edge */
        for (int32_t i = 0; i < m; ++i) cand[i] = i;
        for (int32_t i = m - 1; i > 0; --i) {
            int32_t j = (int32_t)(wl_draw(seed, 3, 0xFFFFFFFFull, (uint64_t)i) % (uint64_t)(i + 1));
            int32_t tmp = cand[i]; cand[i] = cand[j]; cand[j] = tmp;
        }
        for (int32_t i = 0; i < m; ++i) cap[i] = (int32_t)base;
        for (int64_t q = 0; q < rem; ++q) cap[cand[q]] += 1;
        coff[0] = 0;
        for (int32_t i = 0; i < m; ++i) coff[i + 1] = coff[i] + cap[i];
    }
    for (int32_t i = 0; i < m; ++i) cmark[i] = 0;
    for (int32_t j = 0; j < n; ++j) smark[j] = 0;
    int32_t stamp = 0;
    uint64_t tie_ctr = 0;

    for (int32_t j = 0; j < n && status == 0; ++j) {
        for (int32_t e = 0; e < dv; ++e) {
            int32_t ncand = 0;
            ++stamp;
            if (e > 0) {
                /* Expand the current Tanner graph breadth-first from symbol j,
                 * recording the depth at which every check is first reached;
                 * stop when the reached set stops growing or covers all checks. */
                int32_t nsq = 1, nreached = 0, depth = 0;
                sq[0] = j;
                smark[j] = stamp;
                for (;;) {
                    int32_t ncq = 0;
                    for (int32_t a = 0; a < nsq; ++a) {
                        int32_t v = sq[a];
                        for (int32_t b = 0; b < sdeg[v]; ++b) {
                            int32_t c = sadj[(int64_t)v * dv + b];
                            if (cmark[c] != stamp) { cmark[c] = stamp; cdepth[c] = depth; cq[ncq++] = c; }
                        }
                    }
                    nreached += ncq;
                    if (ncq == 0 || nreached == m) break;
                    int32_t nsq2 = 0;
                    for (int32_t a = 0; a < ncq; ++a) {
                        int32_t c = cq[a];
                        for (int32_t b = coff[c]; b < coff[c] + cdeg[c]; ++b) {
                            int32_t v = cadj[b];
                            if (smark[v] != stamp) { smark[v] = stamp; sq2[nsq2++] = v; }
                        }
                    }
                    if (nsq2 == 0) break;
                    int32_t* t = sq; sq = sq2; sq2 = t;
                    nsq = nsq2;
                    ++depth;
                }
            }
            /* Candidates: checks with spare capacity, not adjacent to j (depth 0),
             * at the largest distance from j (unreached counts as infinite).  With
             * capacity to spare this is the PEG rule; otherwise it keeps the new
             * cycle as long as possible. */
            int32_t best = -1;
            for (int32_t i = 0; i < m; ++i) {
                if (cdeg[i] >= cap[i]) continue;
                int32_t dist = (cmark[i] == stamp) ? cdepth[i] : 0x7FFFFFFF;
                if (dist == 0) continue;
                if (dist > best) { best = dist; ncand = 0; }
                if (dist == best) cand[ncand++] = i;
            }
            if (ncand == 0) { status = -2; break; }
            /* lowest current degree among the candidates, ties by a seeded draw */
            int32_t mind = 0x7FFFFFFF;
            for (int32_t a = 0; a < ncand; ++a) if (cdeg[cand[a]] < mind) mind = cdeg[cand[a]];
            int32_t nmin = 0;
            for (int32_t a = 0; a < ncand; ++a) if (cdeg[cand[a]] == mind) cand[nmin++] = cand[a];
            int32_t pick = cand[wl_draw(seed, 3, (uint64_t)j, tie_ctr++) % (uint64_t)nmin];
            sadj[(int64_t)j * dv + sdeg[j]++] = pick;
            cadj[coff[pick] + cdeg[pick]++] = j;
        }
    }
    if (status == 0) {
        for (int32_t i = 0; i < m; ++i)
            if (cdeg[i] != cap[i]) { status = -2; break; }
    }
    if (status == 0) remove_4cycles(n, m, dv, seed, sadj, coff, cdeg, cadj);
    if (status == 0) {
        row_ptr[0] = 0;
        for (int32_t i = 0; i < m; ++i) {
            int32_t* r = cadj + coff[i];
            int32_t d = cdeg[i];
            for (int32_t a = 1; a < d; ++a) {        /* rows are short: insertion sort */
                int32_t v = r[a], b = a - 1;
                while (b >= 0 && r[b] > v) { r[b + 1] = r[b]; --b; }
                r[b + 1] = v;
            }
            memcpy(col_idx + row_ptr[i], r, sizeof(int32_t) * d);
            row_ptr[i + 1] = row_ptr[i] + d;
        }
    }
done:
    free(cap); free(cdeg); free(coff); free(cadj); free(sadj); free(sdeg);
    free(cmark); free(smark); free(sq); free(sq2); free(cq); free(cand); free(cdepth);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Frames: information bits -> systematic codeword -> BPSK -> AWGN            */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t n, k, r;
    const int32_t* info_pos;   /* [k] codeword positions of information bits */
    const int32_t* pivot_pos;  /* [r] codeword positions of parity bits */
    const uint64_t* pmask;     /* [r][kw] info-bit masks, kw = ceil(k/64) */
    double sigma;
    uint64_t seed, frame_offset;
    int64_t f0, f1;
    float* y;                  /* [F][n] */
    uint8_t* cw;               /* [F][ceil(n/8)], LSB-first, bit 1 <=> c = 1 */
    int noiseless;
} frame_job;

static void* frame_worker(void* arg) {
    frame_job* J = (frame_job*)arg;
    const int32_t kw = (J->k + 63) / 64;
    const int32_t nb = (J->n + 7) / 8;
    uint64_t* info = (uint64_t*)malloc(sizeof(uint64_t) * (kw > 0 ? kw : 1));
    uint8_t* c = (uint8_t*)malloc((size_t)J->n);
    for (int64_t f = J->f0; f < J->f1; ++f) {
        const uint64_t fid = J->frame_offset + (uint64_t)f;
        for (int32_t w = 0; w < kw; ++w) info[w] = wl_draw(J->seed, 1, fid, (uint64_t)w);
        if (J->k % 64) info[kw - 1] &= (~0ull) >> (64 - J->k % 64);
        for (int32_t a = 0; a < J->k; ++a) c[J->info_pos[a]] = (uint8_t)((info[a >> 6] >> (a & 63)) & 1u);
        for (int32_t p = 0; p < J->r; ++p) {
            const uint64_t* mk = J->pmask + (int64_t)p * kw;
            uint64_t acc = 0;
            for (int32_t w = 0; w < kw; ++w) acc ^= mk[w] & info[w];
            c[J->pivot_pos[p]] = (uint8_t)(__builtin_popcountll(acc) & 1);
        }
        uint8_t* cwf = J->cw + f * (int64_t)nb;
        memset(cwf, 0, (size_t)nb);
        for (int32_t t = 0; t < J->n; ++t) cwf[t >> 3] |= (uint8_t)(c[t] << (t & 7));
        float* yf = J->y + f * (int64_t)J->n;
        for (int32_t t = 0; t < J->n; t += 2) {
            double z0 = 0.0, z1 = 0.0;
            if (!J->noiseless) {
                uint64_t h0 = wl_draw(J->seed, 2, fid, (uint64_t)t);
                uint64_t h1 = wl_draw(J->seed, 2, fid, (uint64_t)t + 1);
                double u0 = ((double)(h0 >> 11) + 0.5) * 0x1.0p-53;
                double u1 = ((double)(h1 >> 11) + 0.5) * 0x1.0p-53;
                double rad = sqrt(-2.0 * log(u0));
                z0 = rad * cos(6.283185307179586 * u1);
                z1 = rad * sin(6.283185307179586 * u1);
            }
            yf[t] = (float)((1.0 - 2.0 * c[t]) + J->sigma * z0);
            if (t + 1 < J->n) yf[t + 1] = (float)((1.0 - 2.0 * c[t + 1]) + J->sigma * z1);
        }
    }
    free(info); free(c);
    return NULL;
}

/*
 * Fills y[F][n] (FP32 channel samples) and cw[F][ceil(n/8)] (transmitted
 * codeword bits) for frames frame_offset .. frame_offset + F - 1.
 * sigma < 0 produces noiseless frames y = 1 - 2c.  Returns 0 or -1.
 */
int wl_frames(int32_t n, int32_t k, int32_t r, const int32_t* info_pos, const int32_t* pivot_pos,
              const uint64_t* pmask, int64_t n_frames, double sigma, uint64_t seed,
              uint64_t frame_offset, int32_t n_threads, float* y, uint8_t* cw) {
    if (n <= 0 || k < 0 || r < 0 || k + r != n || n_frames < 0) return -1;
    if (n_threads <= 0) n_threads = 1;
    if (n_threads > 256) n_threads = 256;
    if (n_frames < n_threads) n_threads = n_frames > 0 ? (int32_t)n_frames : 1;
    pthread_t th[256];
    frame_job jobs[256];
    for (int32_t i = 0; i < n_threads; ++i) {
        frame_job* J = &jobs[i];
        J->n = n; J->k = k; J->r = r;
        J->info_pos = info_pos; J->pivot_pos = pivot_pos; J->pmask = pmask;
        J->sigma = sigma < 0 ? 0.0 : sigma;
        J->noiseless = sigma < 0;
        J->seed = seed; J->frame_offset = frame_offset;
        J->f0 = n_frames * i / n_threads;
        J->f1 = n_frames * (i + 1) / n_threads;
        J->y = y; J->cw = cw;
    }
    for (int32_t i = 1; i < n_threads; ++i) pthread_create(&th[i], NULL, frame_worker, &jobs[i]);
    frame_worker(&jobs[0]);
    for (int32_t i = 1; i < n_threads; ++i) pthread_join(th[i], NULL);
    return 0;
}
