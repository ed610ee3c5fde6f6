/*
 * gen.c -- seeded synthetic connectivity for the SNN workloads.
 *
 * This is input data, shared by the oracle-side tests and the CUDA path: it
 * holds none of the simulation's arithmetic.  It writes, per network
 * instance, out-edge rows (CSR) whose targets are sorted ascending within a
 * row (sorted rows, Section III-A-2), with no autapses and no multi-edges
 * (Section III-A-2: the graph holds single edges only).
 *
 * Two recipes:
 *   - Bernoulli: every ordered pair (j, i), j != i, is an edge with
 *     probability p (Vogels-Abbott's random connectivity);
 *   - fixed in-degree: every neuron i draws k_exc distinct excitatory and
 *     k_inh distinct inhibitory presynaptic neurons (Brunel's C_E / C_I).
 * Random numbers: xoshiro256** seeded by splitmix64 from (seed, instance,
 * neuron), so every row or column is reproducible on its own.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    uint64_t s[4];
} rng_t;

static uint64_t splitmix64(uint64_t* x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static void rng_seed(rng_t* r, uint64_t seed, uint64_t inst, uint64_t neuron, uint64_t stream)
{
    uint64_t x = seed * 0x100000001B3ULL ^ (inst << 40) ^ (stream << 58) ^ neuron;
    x = splitmix64(&x) ^ neuron;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64(&x);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static inline uint64_t rng_next(rng_t* r)
{
    uint64_t* s = r->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* unbiased integer in [0, m), m >= 1 (Lemire's multiply-and-reject) */
static inline uint32_t rng_below(rng_t* r, uint32_t m)
{
    uint64_t x = (rng_next(r) >> 32) * (uint64_t)m;
    uint32_t lo = (uint32_t)x;
    if (lo < m) {
        uint32_t thresh = (uint32_t)(-m) % m;
        while (lo < thresh) {
            x = (rng_next(r) >> 32) * (uint64_t)m;
            lo = (uint32_t)x;
        }
    }
    return (uint32_t)(x >> 32);
}

static inline double rng_u01(rng_t* r) { return ((rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

/* ---------------- Bernoulli rows ---------------- */

/* Row j of a Bernoulli(p) graph over local ids [0, n): calls emit(i) for
 * every target in ascending order.  Geometric skipping. */
#define BERNOULLI_ROW(seed, inst, n, p, j, EMIT)                             \
    do {                                                                     \
        rng_t r_;                                                            \
        rng_seed(&r_, seed, inst, j, 1);                                     \
        double lq_ = log1p(-(p));                                            \
        int64_t i_ = -1;                                                     \
        for (;;) {                                                           \
            double g_ = floor(log(rng_u01(&r_)) / lq_);                      \
            if (g_ > (double)(n)) break;                                     \
            i_ += 1 + (int64_t)g_;                                           \
            if (i_ >= (int64_t)(n) - 1) break;                               \
            /* candidates skip j itself: candidate c maps to c + (c >= j) */ \
            uint32_t tgt_ = (uint32_t)i_ + ((uint32_t)i_ >= (j) ? 1u : 0u);  \
            EMIT;                                                            \
        }                                                                    \
    } while (0)

uint64_t gen_bernoulli_count(uint64_t seed, uint32_t inst, uint32_t n, double p)
{
    if (n < 2 || !(p > 0.0)) return 0;
    uint64_t total = 0;
    for (uint32_t j = 0; j < n; ++j) {
        if (p >= 1.0) { total += n - 1; continue; }
        BERNOULLI_ROW(seed, inst, n, p, j, (void)tgt_; total++);
    }
    return total;
}

/* row_off: n+1 entries, written as edge_base + local offset; tgt gets
 * global ids (base + local). */
void gen_bernoulli_fill(uint64_t seed, uint32_t inst, uint32_t n, double p, uint32_t base,
                        uint64_t edge_base, uint64_t* row_off, uint32_t* tgt)
{
    uint64_t e = 0;
    for (uint32_t j = 0; j < n; ++j) {
        row_off[j] = edge_base + e;
        if (n < 2 || !(p > 0.0)) continue;
        if (p >= 1.0) {
            for (uint32_t i = 0; i < n; ++i)
                if (i != j) tgt[e++] = base + i;
            continue;
        }
        BERNOULLI_ROW(seed, inst, n, p, j, tgt[e++] = base + tgt_);
    }
    row_off[n] = edge_base + e;
}

/* ---------------- fixed in-degree ---------------- */

/* Draw k distinct ids from [lo, hi) \ {self} into out (unsorted). */
static void draw_distinct(rng_t* r, uint32_t lo, uint32_t hi, uint32_t self, uint32_t k, uint32_t* out,
                          uint64_t* bitmap)
{
    uint32_t m = hi - lo;
    int self_in = (self >= lo && self < hi);
    uint32_t avail = m - (self_in ? 1u : 0u);
    if (k == 0) return;
    if (k > avail) k = avail; /* caller validated; defensive */
    if ((uint64_t)k * 4 <= avail) {
        uint32_t got = 0;
        while (got < k) {
            uint32_t c = lo + rng_below(r, m);
            if (c == self) continue;
            uint32_t b = c - lo;
            if (bitmap[b >> 6] >> (b & 63) & 1) continue;
            bitmap[b >> 6] |= 1ULL << (b & 63);
            out[got++] = c;
        }
        for (uint32_t q = 0; q < k; ++q) {
            uint32_t b = out[q] - lo;
            bitmap[b >> 6] &= ~(1ULL << (b & 63));
        }
    } else {
        /* selection sampling (Knuth, TAOCP 3.4.2, Algorithm S) */
        uint32_t need = k, left = avail, got = 0;
        for (uint32_t c = lo; c < hi && need; ++c) {
            if (c == self) continue;
            if (rng_below(r, left) < need) {
                out[got++] = c;
                --need;
            }
            --left;
        }
    }
}

typedef struct {
    uint64_t seed;
    uint32_t inst, n, n_exc, k_exc, k_inh, base;
    uint32_t i0, i1; /* post range of this worker */
    uint32_t* count; /* per-source counts of this worker (n) */
    uint64_t* pos;   /* per-source write positions of this worker (n) */
    uint32_t* tgt;
    int pass;
} fid_job;

static void* fid_worker(void* arg)
{
    fid_job* J = (fid_job*)arg;
    uint64_t* bitmap = (uint64_t*)calloc(((size_t)J->n + 63) / 64 + 1, sizeof(uint64_t));
    uint32_t* srcs = (uint32_t*)malloc(((size_t)J->k_exc + J->k_inh + 1) * sizeof(uint32_t));
    if (!bitmap || !srcs) { free(bitmap); free(srcs); return (void*)1; }
    for (uint32_t i = J->i0; i < J->i1; ++i) {
        rng_t r;
        rng_seed(&r, J->seed, J->inst, i, 2);
        draw_distinct(&r, 0, J->n_exc, i, J->k_exc, srcs, bitmap);
        draw_distinct(&r, J->n_exc, J->n, i, J->k_inh, srcs + J->k_exc, bitmap);
        uint32_t k = J->k_exc + J->k_inh;
        if (J->pass == 0) {
            for (uint32_t q = 0; q < k; ++q) J->count[srcs[q]]++;
        } else {
            for (uint32_t q = 0; q < k; ++q) J->tgt[J->pos[srcs[q]]++] = J->base + i;
        }
    }
    free(bitmap);
    free(srcs);
    return NULL;
}

/* Fixed in-degree graph of one instance.  row_off: n+1, tgt: n*(k_exc+k_inh).
 * Returns 0, or -1 on bad arguments / allocation failure. */
int gen_fixed_indegree(uint64_t seed, uint32_t inst, uint32_t n, uint32_t n_exc, uint32_t k_exc,
                       uint32_t k_inh, uint32_t base, uint64_t edge_base, uint64_t* row_off, uint32_t* tgt,
                       int threads)
{
    if (n_exc > n) return -1;
    if (k_exc > 0 && k_exc + 1 > n_exc) return -1;
    if (k_inh > 0 && k_inh + 1 > n - n_exc) return -1;
    uint64_t work = (uint64_t)n * (k_exc + k_inh);
    int T = threads < 1 ? 1 : threads;
    if (work < (1u << 22)) T = 1;
    if ((uint32_t)T > n) T = n ? (int)n : 1;
    fid_job* jobs = (fid_job*)calloc(T, sizeof(fid_job));
    pthread_t* th = (pthread_t*)calloc(T, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -1; }
    int rc = 0;
    for (int w = 0; w < T; ++w) {
        fid_job* J = &jobs[w];
        J->seed = seed; J->inst = inst; J->n = n; J->n_exc = n_exc;
        J->k_exc = k_exc; J->k_inh = k_inh; J->base = base; J->tgt = tgt;
        J->i0 = (uint32_t)((uint64_t)n * w / T);
        J->i1 = (uint32_t)((uint64_t)n * (w + 1) / T);
        J->count = (uint32_t*)calloc((size_t)n + 1, sizeof(uint32_t));
        J->pos = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
        if (!J->count || !J->pos) rc = -1;
    }
    if (rc == 0) {
        for (int pass = 0; pass < 2 && rc == 0; ++pass) {
            if (pass == 1) {
                /* rows ordered by source; inside a row, worker w's targets
                 * (posts i0..i1, ascending) follow those of workers < w */
                uint64_t e = 0;
                for (uint32_t j = 0; j < n; ++j) {
                    row_off[j] = edge_base + e;
                    for (int w = 0; w < T; ++w) {
                        jobs[w].pos[j] = e;
                        e += jobs[w].count[j];
                    }
                }
                row_off[n] = edge_base + e;
            }
            for (int w = 0; w < T; ++w) {
                jobs[w].pass = pass;
                if (T == 1) {
                    if (fid_worker(&jobs[w])) rc = -1;
                } else if (pthread_create(&th[w], NULL, fid_worker, &jobs[w])) {
                    rc = -1;
                }
            }
            if (T > 1)
                for (int w = 0; w < T; ++w) {
                    void* ret = NULL;
                    pthread_join(th[w], &ret);
                    if (ret) rc = -1;
                }
        }
    }
    for (int w = 0; w < T; ++w) {
        free(jobs[w].count);
        free(jobs[w].pos);
    }
    free(jobs);
    free(th);
    return rc;
}

/* Weights by source population: rows [row0, row0+n) of one instance get
 * w_exc for local sources < n_exc and w_inh otherwise (lattice units). */
void gen_fill_weights(const uint64_t* row_off, uint32_t n, uint32_t n_exc, int32_t w_exc, int32_t w_inh,
                      int32_t* w)
{
    for (uint32_t j = 0; j < n; ++j) {
        int32_t v = j < n_exc ? w_exc : w_inh;
        for (uint64_t e = row_off[j]; e < row_off[j + 1]; ++e) w[e] = v;
    }
}

/* ------------------------------------------------------------------------
 * Row weights: out[j] = the weight every synapse of row j carries (0 for an
 * empty row).  Returns 1 when every row carries one weight, else 0 (out is
 * then incomplete).  Rows are split among `threads` workers.
 * ---------------------------------------------------------------------- */
typedef struct {
    const uint64_t* row_off;
    const int32_t* w;
    int32_t* out;
    uint32_t j0, j1;
    int ok;
} rw_job;

static void* rw_worker(void* arg)
{
    rw_job* J = (rw_job*)arg;
    J->ok = 1;
    for (uint32_t j = J->j0; j < J->j1; ++j) {
        const uint64_t b = J->row_off[j], e = J->row_off[j + 1];
        const int32_t x = b < e ? J->w[b] : 0;
        for (uint64_t k = b + 1; k < e; ++k)
            if (J->w[k] != x) {
                J->ok = 0;
                return NULL;
            }
        J->out[j] = x;
    }
    return NULL;
}

int gen_row_weights(const uint64_t* row_off, uint32_t n, const int32_t* w, int32_t* out, int threads)
{
    const uint32_t T = threads < 1 ? 1u : (uint32_t)threads;
    rw_job* jobs = (rw_job*)calloc(T, sizeof(rw_job));
    pthread_t* th = (pthread_t*)calloc(T, sizeof(pthread_t));
    int* started = (int*)calloc(T, sizeof(int));
    if (!jobs || !th || !started) {
        free(jobs);
        free(th);
        free(started);
        return 0;
    }
    for (uint32_t t = 0; t < T; ++t) {
        jobs[t].row_off = row_off;
        jobs[t].w = w;
        jobs[t].out = out;
        jobs[t].j0 = (uint32_t)((uint64_t)n * t / T);
        jobs[t].j1 = (uint32_t)((uint64_t)n * (t + 1) / T);
        if (t > 0 && pthread_create(&th[t], NULL, rw_worker, &jobs[t]) == 0) started[t] = 1;
    }
    rw_worker(&jobs[0]);
    int ok = jobs[0].ok;
    for (uint32_t t = 1; t < T; ++t) {
        if (started[t])
            pthread_join(th[t], NULL);
        else
            rw_worker(&jobs[t]);
        ok = ok && jobs[t].ok;
    }
    free(jobs);
    free(th);
    free(started);
    return ok;
}
