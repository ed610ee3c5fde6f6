/*
 * snn_oracle.c -- the plain CPU oracle for the work-queue SNN timestep.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this file.  The product (the CUDA
 * library under paper_1912_07423_b300/) never calls it and shares no code,
 * header, table or constant generator with it.
 *
 * What it computes: a clock-driven simulation of a directed graph of LIF
 * neurons (Section III-A-1, Fig. 1).  Each step t
 *   (1) "Update Neurons" advances every neuron and collects the ids of the
 *       neurons that spike into the spike queue S_t,
 *   (2) with plasticity, "Update Synapses" advances the synapses using the
 *       presynaptic spikes S_{t-d} and the postsynaptic spikes S_t,
 *   (3) "Receive Spikes" delivers the spikes of S_{t-d+1} (the delay FIFO of
 *       d queues) along each spiker's out-edge row into the input
 *       accumulators of the postsynaptic neurons.
 * It is written as that definition, eagerly, one neuron and one edge at a
 * time, with no blocking, fusion or reordering.  The lazy synapse update of
 * Section III-A-1 replays the same per-step updates later, in a batch, so it
 * reaches the eager values and the eager form is the oracle.
 *
 * Precision.  The neuron update is an IEEE binary32 op sequence, one rounding
 * per written operation (compile with -ffp-contract=off and SSE2 math, no
 * fast-math), because the data-parallel path is required to reproduce the
 * spike raster and the membrane state bit for bit.  Synaptic input is
 * integer: weights are int32 multiples of 2^-16 mV and the accumulators sum
 * them exactly (int64 here, checked to fit int32).  orc_run_f64 is a second,
 * independent variant in binary64 with unquantised weights; it only serves
 * statistical comparisons (population rate, ISI CV).
 *
 * Readings of the paper (which defers the model equations to another work):
 *   - Vogels-Abbott CUBA (Section IV): at step t the input that arrived is
 *     added to the synaptic currents ge/gi, the membrane is integrated over
 *     one step with ge/gi held constant, then ge/gi decay:
 *        ge += acc_e*2^-16 ; gi += acc_i*2^-16
 *        if r>0: r -= 1 ; V = V_reset
 *        else:   u = E_L + (ge + gi) ; V = u + (V - u)*Pm
 *        ge *= Pe ; gi *= Pi
 *        if r==0 and V >= V_th: spike, V = V_reset, r = R
 *     The input channel (ge or gi) is the source neuron's population.
 *   - Brunel (Section IV): delta synapses, external Poisson drive of mean
 *     lambda spikes per step of jext lattice units each:
 *        if r>0: r -= 1 ; V = V_reset          (input is discarded)
 *        else:   I = acc + n_ext*jext ; V = V*Pm + I*2^-16
 *                if V >= theta: spike, V = V_reset, r = R
 *   - Poisson: n_ext = #{k : T_k <= u}, T_k = floor(CDF_lambda(k) * 2^32)
 *     for the k whose threshold stays below 2^32 - 1 (CDF summed from the
 *     pmf recursion p_k = p_{k-1} lambda / k in binary64), u one 32-bit
 *     Philox word per neuron per step.
 *   - Random words: Philox4x64-10 (Salmon et al., SC'11), key = (seed,
 *     instance; a problem may start its instance count at inst_key0 so that
 *     one network of a batch can be re-run alone), counter = (local_neuron >> 3, step, tag, 0); the word for a
 *     neuron is 32-bit half (local & 7) of the 256-bit block, low half first.
 *     tag 0 draws the initial potential (step 0), tag 1 the Poisson drive.
 *   - Initial state: V0 = v0_lo + v0_span*u01, u01 = (word >> 8)*2^-24.
 *   - STDP (pair-based, additive, exc->exc synapses), per step t after the
 *     neuron update, in this order: all traces decay (x *= P+, y *= P-);
 *     x_j += 1 for every j in S_{t-d} (the presynaptic spike reaches its
 *     synapses); depression w += rint(Am*y_i) for those rows; y_i += 1 for
 *     i in S_t; potentiation w += rint(Ap*x_j) for the in-edges of i in
 *     S_t; each change is clipped to [0, w_max].  Ap = a_plus*w_max and
 *     Am = a_minus*w_max are rounded to binary32 once.
 *
 * Adjacency construction (Section III-A-2, Fig. 2), a separate function: a
 * job (n, a, b, o) writes n sorted, unique, uniformly distributed random
 * integers from [a, b) at offset o.  Readings: the figure draws n + 2
 * uniforms but the last one's spacing is never used (its running sum is
 * exclusive: it starts at 0 and ends at the normaliser), so n + 1 spacings
 * are drawn; the scale is b - a - n (the figure's "b - n" with a = 0), so
 * that adding a and 0 .. n-1 keeps the values in [a, b); spacings are held
 * as integers (2^-22 units of the binary32 -ln u) so that running sums do
 * not depend on their order, the normalise-and-scale step multiplies by one
 * binary32 factor M / total, and the logarithm is this file's own (range
 * reduction and the atanh series by Horner's rule), so that both sides
 * round every decision the same way.  The figure's row (d) does not follow from its row
 * (c) at two positions (2.32/3.88 printed as 0.4, 2.53/3.88 as 0.6); the
 * tests pin its other steps.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "snn_oracle.h"

/* ------------------------------------------------------------------ */
/* Philox4x64-10, from its published definition (Salmon, Moraes, Dror, */
/* Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11).        */
/* ------------------------------------------------------------------ */
#define PHILOX_M0 0xD2E7470EE14C6C93ULL
#define PHILOX_M1 0xCA5A826395121157ULL
#define PHILOX_W0 0x9E3779B97F4A7C15ULL /* golden ratio */
#define PHILOX_W1 0xBB67AE8584CAA73BULL /* sqrt(3) - 1 */

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    uint64_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += PHILOX_W0;
            k1 += PHILOX_W1;
        }
        unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * c0;
        unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

uint32_t orc_rand_word(uint64_t seed, uint64_t inst, uint64_t local, uint64_t step, uint64_t tag)
{
    uint64_t ctr[4] = {local >> 3, step, tag, 0};
    uint64_t key[2] = {seed, inst};
    uint64_t out[4];
    orc_philox4x64_10(ctr, key, out);
    uint32_t w = (uint32_t)(local & 7);
    return (uint32_t)(out[w >> 1] >> (32 * (w & 1)));
}

/* ------------------------------------------------------------------ */
/* Poisson sampling by integer CDF thresholds.                          */
/* ------------------------------------------------------------------ */
int orc_poisson_table(double lambda, uint32_t* T, int cap)
{
    if (!(lambda >= 0.0)) return -1;
    double p = exp(-lambda); /* P(X = 0) */
    double cdf = p;
    int n = 0;
    for (int k = 0;; ++k) {
        if (k > 0) {
            p = p * lambda / (double)k;
            cdf = cdf + p;
        }
        double s = floor(cdf * 4294967296.0);
        /* stop once a threshold would reach 2^32 - 1: from there on the
         * partial sums only repeat it, and the tail left is below 2^-31 */
        if (s >= 4294967295.0) break;
        if (n == cap) return -2;
        T[n++] = (uint32_t)s;
        if (k > 100000) return -3;
    }
    return n;
}

uint32_t orc_poisson_sample(const uint32_t* T, int n, uint32_t u)
{
    uint32_t k = 0;
    for (int i = 0; i < n; ++i)
        if (T[i] <= u) ++k;
    return k;
}

/* ------------------------------------------------------------------ */
/* Receive Spikes: deliver every spike of a queue along its row.        */
/* ------------------------------------------------------------------ */
static int channel_of(const orc_problem* P, uint32_t j)
{
    if (P->model != ORC_VOGELS) return 0;
    for (uint32_t b = 0; b < P->n_inst; ++b)
        if (j >= P->inst_off[b] && j < P->inst_off[b + 1])
            return (j - P->inst_off[b]) >= P->params[b].n_exc ? 1 : 0;
    return 0;
}

int orc_receive(const orc_problem* P, const int32_t* w, const uint32_t* spikes, uint64_t n_spikes,
                int64_t* acc0, int64_t* acc1, uint64_t* events)
{
    for (uint64_t s = 0; s < n_spikes; ++s) {
        uint32_t j = spikes[s];
        int64_t* acc = channel_of(P, j) ? acc1 : acc0;
        for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e) {
            acc[P->tgt[e]] += w[e];
            if (acc[P->tgt[e]] > INT32_MAX || acc[P->tgt[e]] < INT32_MIN) return ORC_E_RANGE;
        }
        *events += P->row_off[j + 1] - P->row_off[j];
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Growable spike log (the raster).  Spikes of step t are the slice     */
/* [step_start[t], step_start[t+1]); the delay FIFO reads old slices.   */
/* ------------------------------------------------------------------ */
typedef struct {
    uint32_t* step;
    uint32_t* id;
    uint64_t n, cap;
} spike_log;

static int log_push(spike_log* L, uint32_t t, uint32_t id)
{
    if (L->n == L->cap) {
        uint64_t nc = L->cap ? 2 * L->cap : 4096;
        uint32_t* s = (uint32_t*)realloc(L->step, nc * sizeof(uint32_t));
        if (!s) return ORC_E_NOMEM;
        L->step = s;
        uint32_t* i = (uint32_t*)realloc(L->id, nc * sizeof(uint32_t));
        if (!i) return ORC_E_NOMEM;
        L->id = i;
        L->cap = nc;
    }
    L->step[L->n] = t;
    L->id[L->n] = id;
    L->n++;
    return ORC_OK;
}

/* Per-instance binary32 constants, each the binary64 value rounded once. */
typedef struct {
    float Pm, Pe, Pi, Pp, Pn, Ap, Am;
    float v_th, v_reset, e_l, v0_lo, v0_span;
    uint32_t T[ORC_POISSON_CAP];
    int nT;
} inst_consts;

static int make_consts(const orc_params* p, inst_consts* c)
{
    c->Pm = (float)exp(-p->dt / p->tau_m);
    c->Pe = (float)(p->tau_e > 0 ? exp(-p->dt / p->tau_e) : 0.0);
    c->Pi = (float)(p->tau_i > 0 ? exp(-p->dt / p->tau_i) : 0.0);
    c->Pp = (float)(p->tau_plus > 0 ? exp(-p->dt / p->tau_plus) : 0.0);
    c->Pn = (float)(p->tau_minus > 0 ? exp(-p->dt / p->tau_minus) : 0.0);
    c->Ap = (float)(p->a_plus * (double)p->w_max_q);
    c->Am = (float)(p->a_minus * (double)p->w_max_q);
    c->v_th = (float)p->v_th;
    c->v_reset = (float)p->v_reset;
    c->e_l = (float)p->e_l;
    c->v0_lo = (float)p->v0_lo;
    c->v0_span = (float)p->v0_span;
    c->nT = orc_poisson_table(p->lambda, c->T, ORC_POISSON_CAP);
    return c->nT < 0 ? ORC_E_ARG : ORC_OK;
}

static int check_problem(const orc_problem* P)
{
    if (P->n_inst == 0 || P->delay < 1) return ORC_E_ARG;
    if (P->model != ORC_VOGELS && P->model != ORC_BRUNEL) return ORC_E_ARG;
    if (P->inst_off[0] != 0) return ORC_E_ARG;
    for (uint32_t b = 0; b < P->n_inst; ++b) {
        if (P->inst_off[b + 1] < P->inst_off[b]) return ORC_E_ARG;
        if (P->params[b].n_exc > P->inst_off[b + 1] - P->inst_off[b]) return ORC_E_ARG;
    }
    uint32_t N = P->inst_off[P->n_inst];
    if (P->row_off[0] != 0) return ORC_E_ARG;
    for (uint32_t j = 0; j < N; ++j)
        if (P->row_off[j + 1] < P->row_off[j]) return ORC_E_ARG;
    for (uint32_t b = 0; b < P->n_inst; ++b)
        for (uint32_t j = P->inst_off[b]; j < P->inst_off[b + 1]; ++j)
            for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e)
                if (P->tgt[e] < P->inst_off[b] || P->tgt[e] >= P->inst_off[b + 1]) return ORC_E_ARG;
    return ORC_OK;
}

static int is_exc(const orc_problem* P, uint32_t b, uint32_t i)
{
    return i - P->inst_off[b] < P->params[b].n_exc;
}

static uint32_t inst_of(const orc_problem* P, uint32_t i)
{
    uint32_t b = 0;
    while (i >= P->inst_off[b + 1]) ++b;
    return b;
}

static int32_t clip_w(int64_t w, int32_t w_max)
{
    if (w < 0) return 0;
    if (w > w_max) return w_max;
    return (int32_t)w;
}

/* ------------------------------------------------------------------ */
/* The binary32 oracle.                                                 */
/* ------------------------------------------------------------------ */
int orc_run(const orc_problem* P, orc_state* S, orc_raster* R)
{
    int st = check_problem(P);
    if (st != ORC_OK) return st;
    const uint32_t N = P->inst_off[P->n_inst];
    const uint64_t E = P->row_off[N];
    const uint32_t d = P->delay;
    const float lattice = 1.0f / 65536.0f; /* 2^-16 mV */

    inst_consts* C = (inst_consts*)calloc(P->n_inst, sizeof(inst_consts));
    int64_t* acc0 = (int64_t*)calloc(N ? N : 1, sizeof(int64_t));
    int64_t* acc1 = (int64_t*)calloc(N ? N : 1, sizeof(int64_t));
    uint64_t* step_start = (uint64_t*)calloc((size_t)P->n_steps + 2, sizeof(uint64_t));
    spike_log L = {0};
    /* column index of the plastic synapses (exc -> exc), for potentiation */
    uint64_t* col_off = NULL;
    uint64_t* col_edge = NULL;
    uint32_t* col_pre = NULL;
    if (!C || !acc0 || !acc1 || !step_start) { st = ORC_E_NOMEM; goto done; }
    for (uint32_t b = 0; b < P->n_inst; ++b)
        if ((st = make_consts(&P->params[b], &C[b])) != ORC_OK) goto done;

    /* Init stage: N -> N_0 (Fig. 1 caption).  State may be supplied by the
     * caller (S->init_given), otherwise it is drawn as documented above. */
    if (!S->init_given) {
        for (uint32_t b = 0; b < P->n_inst; ++b)
            for (uint32_t i = P->inst_off[b]; i < P->inst_off[b + 1]; ++i) {
                uint32_t u = orc_rand_word(P->seed, P->inst_key0 + b, i - P->inst_off[b], 0, 0);
                float u01 = (float)(u >> 8) * (1.0f / 16777216.0f);
                float t = C[b].v0_span * u01;
                S->V[i] = C[b].v0_lo + t;
                S->ge[i] = 0.0f;
                S->gi[i] = 0.0f;
                S->r[i] = 0;
                S->x[i] = 0.0f;
                S->y[i] = 0.0f;
                S->acc0[i] = 0;
                S->acc1[i] = 0;
            }
        memcpy(S->w, P->w, E * sizeof(int32_t));
    }
    for (uint32_t i = 0; i < N; ++i) {
        acc0[i] = S->acc0[i];
        acc1[i] = S->acc1[i];
    }

    if (P->stdp) {
        col_off = (uint64_t*)calloc((size_t)N + 1, sizeof(uint64_t));
        if (!col_off) { st = ORC_E_NOMEM; goto done; }
        for (uint32_t b = 0; b < P->n_inst; ++b)
            for (uint32_t j = P->inst_off[b]; j < P->inst_off[b + 1]; ++j)
                if (is_exc(P, b, j))
                    for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e)
                        if (is_exc(P, b, P->tgt[e])) col_off[P->tgt[e] + 1]++;
        for (uint32_t i = 0; i < N; ++i) col_off[i + 1] += col_off[i];
        uint64_t nplastic = col_off[N];
        col_edge = (uint64_t*)malloc((nplastic ? nplastic : 1) * sizeof(uint64_t));
        col_pre = (uint32_t*)malloc((nplastic ? nplastic : 1) * sizeof(uint32_t));
        uint64_t* fill = (uint64_t*)malloc(((size_t)N + 1) * sizeof(uint64_t));
        if (!col_edge || !col_pre || !fill) { free(fill); st = ORC_E_NOMEM; goto done; }
        memcpy(fill, col_off, ((size_t)N + 1) * sizeof(uint64_t));
        for (uint32_t b = 0; b < P->n_inst; ++b)
            for (uint32_t j = P->inst_off[b]; j < P->inst_off[b + 1]; ++j)
                if (is_exc(P, b, j))
                    for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e)
                        if (is_exc(P, b, P->tgt[e])) {
                            uint64_t k = fill[P->tgt[e]]++;
                            col_edge[k] = e;
                            col_pre[k] = j;
                        }
        free(fill);
    }

    uint32_t no = 0; /* next override (overrides are sorted by step) */
    R->events = 0;
    for (uint32_t t = 0; t < P->n_steps; ++t) {
        /* overrides of the membrane potential, applied before the update */
        while (no < P->n_over && P->over_step[no] < t) ++no;
        while (no < P->n_over && P->over_step[no] == t) {
            S->V[P->over_id[no]] = P->over_v[no];
            ++no;
        }

        /* (1) Update Neurons: N_t -> N'_{t+1}, producing S_t (Section III-A-1) */
        step_start[t] = L.n;
        for (uint32_t b = 0; b < P->n_inst; ++b) {
            const inst_consts* c = &C[b];
            const orc_params* p = &P->params[b];
            for (uint32_t i = P->inst_off[b]; i < P->inst_off[b + 1]; ++i) {
                int spike = 0;
                if (P->model == ORC_VOGELS) {
                    float ge = S->ge[i] + (float)(int32_t)acc0[i] * lattice;
                    float gi = S->gi[i] + (float)(int32_t)acc1[i] * lattice;
                    float V = S->V[i];
                    int32_t r = S->r[i];
                    if (r > 0) {
                        r -= 1;
                        V = c->v_reset;
                    } else {
                        float g = ge + gi;
                        float u = c->e_l + g;
                        float dv = V - u;
                        float dvp = dv * c->Pm;
                        V = u + dvp;
                    }
                    ge = ge * c->Pe;
                    gi = gi * c->Pi;
                    if (r == 0 && V >= c->v_th) {
                        spike = 1;
                        V = c->v_reset;
                        r = (int32_t)p->refractory_steps;
                    }
                    S->V[i] = V;
                    S->ge[i] = ge;
                    S->gi[i] = gi;
                    S->r[i] = r;
                } else {
                    float V = S->V[i];
                    int32_t r = S->r[i];
                    if (r > 0) {
                        r -= 1;
                        V = c->v_reset;
                    } else {
                        uint32_t u = orc_rand_word(P->seed, P->inst_key0 + b, i - P->inst_off[b], t, 1);
                        int64_t n_ext = orc_poisson_sample(c->T, c->nT, u);
                        int64_t I = acc0[i] + n_ext * (int64_t)p->jext_q;
                        if (I > INT32_MAX || I < INT32_MIN) { st = ORC_E_RANGE; goto done; }
                        float vd = V * c->Pm;
                        float in = (float)(int32_t)I * lattice;
                        V = vd + in;
                        if (V >= c->v_th) {
                            spike = 1;
                            V = c->v_reset;
                            r = (int32_t)p->refractory_steps;
                        }
                    }
                    S->V[i] = V;
                    S->r[i] = r;
                }
                acc0[i] = 0;
                acc1[i] = 0;
                if (spike && (st = log_push(&L, t, i)) != ORC_OK) goto done;
            }
        }
        step_start[t + 1] = L.n;

        /* (2) Update Synapses: Syn_t -> Syn_{t+1} from S_{t-d} and S_t (Section III-A-1) */
        if (P->stdp) {
            for (uint32_t b = 0; b < P->n_inst; ++b)
                for (uint32_t i = P->inst_off[b]; i < P->inst_off[b + 1]; ++i)
                    if (is_exc(P, b, i)) {
                        S->x[i] = S->x[i] * C[b].Pp;
                        S->y[i] = S->y[i] * C[b].Pn;
                    }
            if (t >= d) {
                uint64_t a0 = step_start[t - d], a1 = step_start[t - d + 1];
                for (uint64_t s = a0; s < a1; ++s) {
                    uint32_t j = L.id[s];
                    uint32_t b = inst_of(P, j);
                    if (is_exc(P, b, j)) S->x[j] = S->x[j] + 1.0f;
                }
                for (uint64_t s = a0; s < a1; ++s) {
                    uint32_t j = L.id[s];
                    uint32_t b = inst_of(P, j);
                    if (!is_exc(P, b, j)) continue;
                    for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e) {
                        uint32_t i = P->tgt[e];
                        if (!is_exc(P, b, i)) continue;
                        float dw = C[b].Am * S->y[i];
                        S->w[e] = clip_w((int64_t)S->w[e] + (int64_t)rintf(dw), P->params[b].w_max_q);
                    }
                }
            }
            for (uint64_t s = step_start[t]; s < step_start[t + 1]; ++s) {
                uint32_t i = L.id[s];
                if (is_exc(P, inst_of(P, i), i)) S->y[i] = S->y[i] + 1.0f;
            }
            for (uint64_t s = step_start[t]; s < step_start[t + 1]; ++s) {
                uint32_t i = L.id[s];
                uint32_t b = inst_of(P, i);
                if (!is_exc(P, b, i)) continue;
                for (uint64_t k = col_off[i]; k < col_off[i + 1]; ++k) {
                    float dw = C[b].Ap * S->x[col_pre[k]];
                    uint64_t e = col_edge[k];
                    S->w[e] = clip_w((int64_t)S->w[e] + (int64_t)rintf(dw), P->params[b].w_max_q);
                }
            }
        }

        /* (3) Receive Spikes: deliver S_{t-d+1} (the FIFO of d queues, Fig. 1) */
        if (t + 1 >= d) {
            uint32_t ts = t + 1 - d;
            st = orc_receive(P, S->w, L.id + step_start[ts], step_start[ts + 1] - step_start[ts], acc0,
                             acc1, &R->events);
            if (st != ORC_OK) goto done;
        }
    }
    for (uint32_t i = 0; i < N; ++i) {
        S->acc0[i] = (int32_t)acc0[i];
        S->acc1[i] = (int32_t)acc1[i];
    }
    R->n = L.n;
    R->step = L.step;
    R->id = L.id;
    L.step = NULL;
    L.id = NULL;

done:
    free(C);
    free(acc0);
    free(acc1);
    free(step_start);
    free(L.step);
    free(L.id);
    free(col_off);
    free(col_edge);
    free(col_pre);
    return st;
}

/* ------------------------------------------------------------------ */
/* The binary64 variant: same pipeline, double state, unquantised       */
/* weights (mV, one per edge), same Poisson draws.  No plasticity.      */
/* ------------------------------------------------------------------ */
int orc_run_f64(const orc_problem* P, const double* w_mV, double* V_out, orc_raster* R)
{
    int st = check_problem(P);
    if (st != ORC_OK) return st;
    if (P->stdp) return ORC_E_ARG;
    const uint32_t N = P->inst_off[P->n_inst];
    const uint32_t d = P->delay;
    double* V = (double*)malloc((N ? N : 1) * sizeof(double));
    double* ge = (double*)calloc(N ? N : 1, sizeof(double));
    double* gi = (double*)calloc(N ? N : 1, sizeof(double));
    double* in0 = (double*)calloc(N ? N : 1, sizeof(double));
    double* in1 = (double*)calloc(N ? N : 1, sizeof(double));
    int32_t* r = (int32_t*)calloc(N ? N : 1, sizeof(int32_t));
    uint64_t* step_start = (uint64_t*)calloc((size_t)P->n_steps + 2, sizeof(uint64_t));
    uint32_t* T = (uint32_t*)malloc((size_t)P->n_inst * ORC_POISSON_CAP * sizeof(uint32_t));
    int* nT = (int*)malloc(P->n_inst * sizeof(int));
    spike_log L = {0};
    if (!V || !ge || !gi || !in0 || !in1 || !r || !step_start || !T || !nT) { st = ORC_E_NOMEM; goto done; }
    for (uint32_t b = 0; b < P->n_inst; ++b) {
        nT[b] = orc_poisson_table(P->params[b].lambda, T + (size_t)b * ORC_POISSON_CAP, ORC_POISSON_CAP);
        if (nT[b] < 0) { st = ORC_E_ARG; goto done; }
        for (uint32_t i = P->inst_off[b]; i < P->inst_off[b + 1]; ++i) {
            uint32_t u = orc_rand_word(P->seed, P->inst_key0 + b, i - P->inst_off[b], 0, 0);
            V[i] = P->params[b].v0_lo + P->params[b].v0_span * ((double)(u >> 8) / 16777216.0);
        }
    }
    R->events = 0;
    for (uint32_t t = 0; t < P->n_steps; ++t) {
        step_start[t] = L.n;
        for (uint32_t b = 0; b < P->n_inst; ++b) {
            const orc_params* p = &P->params[b];
            double Pm = exp(-p->dt / p->tau_m);
            for (uint32_t i = P->inst_off[b]; i < P->inst_off[b + 1]; ++i) {
                int spike = 0;
                if (P->model == ORC_VOGELS) {
                    ge[i] += in0[i];
                    gi[i] += in1[i];
                    if (r[i] > 0) {
                        r[i] -= 1;
                        V[i] = p->v_reset;
                    } else {
                        double u = p->e_l + ge[i] + gi[i];
                        V[i] = u + (V[i] - u) * Pm;
                    }
                    ge[i] *= exp(-p->dt / p->tau_e);
                    gi[i] *= exp(-p->dt / p->tau_i);
                    if (r[i] == 0 && V[i] >= p->v_th) spike = 1;
                } else {
                    if (r[i] > 0) {
                        r[i] -= 1;
                        V[i] = p->v_reset;
                    } else {
                        uint32_t u = orc_rand_word(P->seed, P->inst_key0 + b, i - P->inst_off[b], t, 1);
                        double n_ext = orc_poisson_sample(T + (size_t)b * ORC_POISSON_CAP, nT[b], u);
                        V[i] = V[i] * Pm + in0[i] + n_ext * p->jext_q / 65536.0;
                        if (V[i] >= p->v_th) spike = 1;
                    }
                }
                if (spike) {
                    V[i] = p->v_reset;
                    r[i] = (int32_t)p->refractory_steps;
                    if ((st = log_push(&L, t, i)) != ORC_OK) goto done;
                }
                in0[i] = 0.0;
                in1[i] = 0.0;
            }
        }
        step_start[t + 1] = L.n;
        if (t + 1 >= d) {
            uint32_t ts = t + 1 - d;
            for (uint64_t s = step_start[ts]; s < step_start[ts + 1]; ++s) {
                uint32_t j = L.id[s];
                double* in = channel_of(P, j) ? in1 : in0;
                for (uint64_t e = P->row_off[j]; e < P->row_off[j + 1]; ++e) in[P->tgt[e]] += w_mV[e];
                R->events += P->row_off[j + 1] - P->row_off[j];
            }
        }
    }
    if (V_out) memcpy(V_out, V, N * sizeof(double));
    R->n = L.n;
    R->step = L.step;
    R->id = L.id;
    L.step = NULL;
    L.id = NULL;
done:
    free(V); free(ge); free(gi); free(in0); free(in1); free(r);
    free(step_start); free(T); free(nT);
    free(L.step); free(L.id);
    return st;
}

/* ------------------------------------------------------------------ */
/* Adjacency construction, Fig. 2: sorted random integers by           */
/* exponential spacings.                                                */
/* ------------------------------------------------------------------ */

/* -ln(u) for u in (0, 1], binary32, one operation at a time: u = m 2^e with
 * m in [1, 2) (read from the bits), ln m = 2 atanh(s) = 2 s (1 + s^2/3 +
 * s^4/5 + ... + s^12/13) with s = (m - 1) / (m + 1) < 1/3, the polynomial
 * in s^2 by Horner's rule with binary32 coefficients 1/k, ln u = e ln 2 +
 * ln m. */
float orc_neg_ln(float u)
{
    static const float inv[7] = {1.0f, 1.0f / 3.0f, 1.0f / 5.0f, 1.0f / 7.0f, 1.0f / 9.0f, 1.0f / 11.0f, 1.0f / 13.0f};
    uint32_t bits;
    memcpy(&bits, &u, 4);
    const int32_t e = (int32_t)((bits >> 23) & 0xffu) - 127;
    const uint32_t mb = (bits & 0x7fffffu) | 0x3f800000u;
    float m;
    memcpy(&m, &mb, 4);
    const float s = (m - 1.0f) / (m + 1.0f);
    const float s2 = s * s;
    float p = inv[6];
    for (int k = 5; k >= 0; --k) p = p * s2 + inv[k];
    const float ln_u = (float)e * 0.693147182f + 2.0f * (s * p);
    return -ln_u;
}

/* The steps of one job from its n + 1 uniforms u[0..n] in (0, 1]:
 * exponential spacings E_k = -ln u_k, held as q_k = E_k 2^22 rounded
 * (binary32, then an integer: the sums are exact in any order, and 32 of
 * them fit 32 bits); the exclusive running sums c_0 = 0, c_k = q_0 + ... +
 * q_{k-1} (c_{n+1} the total, which normalises); output k = 1..n:
 * a + round(c_k f) + (k - 1) with f = M / c_{n+1} in binary32, M = b - a - n
 * (the added k - 1 keeps the values distinct; the rounding is half up, at
 * most M).  q and c may be NULL.  Needs n <= b - a and M <= 2^24. */
int orc_job_from_uniforms(const float* u, uint32_t n, uint32_t a, uint32_t b, uint32_t* q, uint64_t* c,
                          uint32_t* out)
{
    if (b < a || n > b - a || b - a - n > (1u << 24)) return ORC_E_ARG;
    const uint32_t M = b - a - n;
    uint64_t* cc = c ? c : (uint64_t*)malloc(((size_t)n + 2) * sizeof(uint64_t));
    if (!cc) return ORC_E_NOMEM;
    cc[0] = 0;
    for (uint32_t k = 0; k <= n; ++k) {
        const uint32_t qk = (uint32_t)(orc_neg_ln(u[k]) * 4194304.0f + 0.5f);
        if (q) q[k] = qk;
        cc[k + 1] = cc[k] + qk;
    }
    const uint64_t total = cc[n + 1];
    const float f = total ? (float)M / (float)total : 0.0f;
    for (uint32_t k = 1; k <= n; ++k) {
        uint32_t r = (uint32_t)((float)cc[k] * f + 0.5f);
        if (r > M) r = M;
        out[k - 1] = a + r + (k - 1);
    }
    if (!c) free(cc);
    return ORC_OK;
}

/* Job j draws its uniforms from Philox4x64-10 with key (seed, j), counter
 * (k >> 3, 0, 2, 0), word k & 7: u_k = (word >> 8 + 1) 2^-24; its n values
 * go to out[0 .. n). */
int orc_expand_job(const orc_job* J, uint64_t j, uint64_t seed, uint32_t* out)
{
    if (J->b < J->a || J->n > J->b - J->a || J->b - J->a - J->n > (1u << 24)) return ORC_E_ARG;
    float* u = (float*)malloc(((size_t)J->n + 1) * sizeof(float));
    if (!u) return ORC_E_NOMEM;
    for (uint32_t k = 0; k <= J->n; ++k)
        u[k] = (float)((orc_rand_word(seed, j, k, 0, 2) >> 8) + 1u) * (1.0f / 16777216.0f);
    const int st = orc_job_from_uniforms(u, J->n, J->a, J->b, NULL, NULL, out);
    free(u);
    return st;
}

int orc_expand_jobs(const orc_job* jobs, uint64_t n_jobs, uint64_t seed, uint32_t* out, uint64_t out_len)
{
    for (uint64_t j = 0; j < n_jobs; ++j) {
        const orc_job J = jobs[j];
        if (J.o > out_len || J.n > out_len - J.o) return ORC_E_ARG;
        const int st = orc_expand_job(&J, j, seed, out + J.o);
        if (st != ORC_OK) return st;
    }
    return ORC_OK;
}

void orc_raster_free(orc_raster* R)
{
    free(R->step);
    free(R->id);
    R->step = NULL;
    R->id = NULL;
    R->n = 0;
}
