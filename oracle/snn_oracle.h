/*
 * snn_oracle.h -- private interface of the CPU oracle (test infrastructure
 * only; see snn_oracle.c).  Nothing in the product includes this header.
 */
#ifndef SNN_ORACLE_H
#define SNN_ORACLE_H
#include <stdint.h>

#define ORC_OK 0
#define ORC_E_ARG -1
#define ORC_E_NOMEM -2
#define ORC_E_RANGE -3 /* an accumulator left the int32 range */

#define ORC_VOGELS 0
#define ORC_BRUNEL 1
#define ORC_POISSON_CAP 64

/* Model constants of one network instance (units: ms, mV, lattice units of
 * 2^-16 mV for the integer fields). */
typedef struct {
    uint32_t n_exc;            /* local ids [0, n_exc) are excitatory */
    uint32_t refractory_steps; /* R */
    int32_t jext_q;            /* Brunel: lattice units per external spike */
    int32_t w_max_q;           /* STDP: upper clip of plastic weights */
    double dt, tau_m, v_th, v_reset;
    double e_l, tau_e, tau_i; /* Vogels CUBA */
    double lambda;            /* Brunel: Poisson mean per step */
    double v0_lo, v0_span;    /* V0 = v0_lo + v0_span * u01 */
    double tau_plus, tau_minus, a_plus, a_minus; /* STDP */
} orc_params;

typedef struct {
    int32_t model; /* ORC_VOGELS or ORC_BRUNEL */
    int32_t stdp;  /* 1: trace STDP on exc -> exc synapses */
    uint32_t n_inst;
    uint32_t delay; /* d >= 1 steps */
    const uint32_t* inst_off; /* n_inst + 1 global neuron offsets */
    const orc_params* params; /* n_inst */
    uint64_t seed;
    const uint64_t* row_off; /* N + 1 */
    const uint32_t* tgt;     /* E, global ids inside the source's instance */
    const int32_t* w;        /* E, lattice units */
    uint32_t n_steps;
    uint32_t n_over; /* membrane overrides, sorted by step */
    const uint32_t* over_step;
    const uint32_t* over_id;
    const float* over_v;
    uint32_t inst_key0; /* Philox key word 1 of instance b is inst_key0 + b */
    uint32_t pad;
} orc_problem;

/* Neuron and synapse state; arrays of N (w: E) owned by the caller. */
typedef struct {
    int32_t init_given; /* 0: the oracle draws N_0 itself and copies w */
    float* V;
    float* ge;
    float* gi;
    int32_t* r;
    float* x;
    float* y;
    int32_t* acc0;
    int32_t* acc1;
    int32_t* w;
} orc_state;

typedef struct {
    uint64_t n;
    uint32_t* step; /* sorted by (step, id) */
    uint32_t* id;
    uint64_t events; /* delivered synaptic events */
} orc_raster;

/* A job of the adjacency construction (Fig. 2): write n sorted, unique,
 * uniformly distributed random integers from [a, b) to out[o .. o + n). */
typedef struct {
    uint32_t n, a, b, reserved;
    uint64_t o;
} orc_job;

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
uint32_t orc_rand_word(uint64_t seed, uint64_t inst, uint64_t local, uint64_t step, uint64_t tag);
int orc_poisson_table(double lambda, uint32_t* T, int cap);
uint32_t orc_poisson_sample(const uint32_t* T, int n, uint32_t u);
int orc_receive(const orc_problem* P, const int32_t* w, const uint32_t* spikes, uint64_t n_spikes,
                int64_t* acc0, int64_t* acc1, uint64_t* events);
int orc_run(const orc_problem* P, orc_state* S, orc_raster* R);
int orc_run_f64(const orc_problem* P, const double* w_mV, double* V_out, orc_raster* R);
float orc_neg_ln(float u);
int orc_job_from_uniforms(const float* u, uint32_t n, uint32_t a, uint32_t b, uint32_t* q, uint64_t* c,
                          uint32_t* out);
int orc_expand_jobs(const orc_job* jobs, uint64_t n_jobs, uint64_t seed, uint32_t* out, uint64_t out_len);
/* One job alone, by its index j in the job list (the index keys its random draws). */
int orc_expand_job(const orc_job* job, uint64_t j, uint64_t seed, uint32_t* out);
void orc_raster_free(orc_raster* R);

#endif
