/*
 * snn.h -- C ABI of the B300 work-queue SNN library (libsnn.so).
 *
 * The library simulates a directed graph of leaky integrate-and-fire
 * neurons, clock-driven, one timestep at a time, and returns its firing
 * pattern.  The problem statement follows the paper: neurons and synapses
 * with weights and a synaptic delay, simulated for T steps, whose output is
 * the spike raster (Section I; Section III-A-1).  One timestep is the
 * paper's pipeline (Fig. 1):
 *   Update Neurons   -- every neuron is advanced from N_t to N'_{t+1}; the
 *                       ids of the neurons that spike go to the spike queue
 *                       S_t (Section III-A-1, III-A-2: an array with an
 *                       atomic insertion index),
 *   delay FIFO       -- S_t waits in a ring of d queues (d+1 with
 *                       plasticity) (Section III-A-1),
 *   Update Synapses  -- with plasticity, pair STDP from S_{t-d} (pre) and
 *                       S_t (post) (Section III-A-1),
 *   Receive Spikes   -- every spike of S_{t-d+1} is delivered along its
 *                       out-edge row into the input accumulators of its
 *                       targets (Section III-A-2: sorted adjacency rows).
 * Many independent networks ("instances") of uneven size are stepped
 * together over one concatenated graph.
 *
 * Units and exactness.  Synaptic weights are int32 multiples of 2^-16 mV
 * (the lattice); input accumulates in int32 in any order with the same
 * result.  The neuron update is a fixed binary32 operation sequence without
 * fused multiply-add, so two runs of the same input give the same raster
 * and state bit for bit.
 *
 * Threading.  A context is used by one host thread at a time.  All device
 * work is enqueued on the stream given at creation; calls that return data
 * to the host synchronise that stream.
 *
 * Errors.  Every call returns an snn_status; no exception crosses the ABI.
 * snn_last_error() gives a one-line description of the last failure.
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct snn_ctx snn_ctx; /* opaque, owned by the library */

typedef enum {
    SNN_OK = 0,
    SNN_E_ARG = -1,      /* invalid argument; nothing was changed */
    SNN_E_NOMEM = -2,    /* a device or host allocation failed */
    SNN_E_CUDA = -3,     /* a CUDA call failed; the context is unusable */
    SNN_E_OVERFLOW = -4, /* the spike log filled up; the simulation itself is intact */
    SNN_E_TIMEOUT = -5,  /* a bounded device-side wait gave up */
    SNN_E_STATE = -6     /* call out of order (e.g. snn_step before snn_build_graph) */
} snn_status;

typedef enum {
    SNN_VOGELS_CUBA = 0, /* LIF with exponential exc/inh currents and constant drive (Section IV) */
    SNN_BRUNEL = 1,      /* LIF with delta synapses and Poisson drive (Section IV) */
    /* Models of the generic update (Section III-B): device functors with init() and update()
     * callbacks compiled into the library from csrc/snn_models.cuh; their per-neuron state is
     * one record (SNN_FIELD_MODEL).  Receive Spikes stays the library's: a neuron's update sees
     * the sum of the weights it received since its last update. */
    SNN_MODEL_RELAY = 2,     /* the paper's tutorial model (Listing 1): a neuron fires at the step
                                after it received input; local ids < n_exc fire at step 0 */
    SNN_MODEL_BRUNEL_LIF = 3 /* Brunel written as a Poisson-driven specialisation of the LIF
                                building block; the values of SNN_BRUNEL, bit for bit */
} snn_model;

/* snn_config.flags */
#define SNN_F_STDP 1u  /* pair STDP on exc -> exc synapses (Brunel only; "Brunel+") */
#define SNN_F_W16 2u   /* weights stored as int16 codes x 2^shift(row); else binary32 */
#define SNN_F_STATS 4u /* keep per-neuron spike counts and ISI moments for snn_stats */
#define SNN_F_UNPACKED 8u /* read the u32 target and int16 code arrays even where a compressed layout
                             applies.  The compressed layouts (SNN_F_W16, no STDP): the tiled receive's
                             packed edges where every instance has at most 65,536 neurons (one u32 per
                             edge, target offset << 16 | code), and the global receive's row weights
                             where every row carries one weight -- the source population's, as in the
                             paper's models (Section III-A-2, Table 2) -- so that it reads the 4-byte
                             targets alone */
#define SNN_F_LAZY 16u /* with SNN_F_STDP: lazy Update Synapses (Section III-A-1).  The plastic
                          synapses of a row are left stale and brought up to date in one pass
                          when the row transmits a spike or when its age reaches the history
                          length lazy_fifo; the weights and traces are the eager rule's, bit for
                          bit (snn_read_state / snn_write_state bring every row up to date first).
                          For the pair rule here the eager form, which touches only the rows of the
                          arriving spikes and the columns of the spiking neurons, measured as fast */
#define SNN_F_SERIAL 32u /* run Update Neurons and Receive Spikes as separate kernels, one after the
                            other.  Without it the library runs both stages of a step in one kernel
                            where that applies (the Brunel model without plasticity, 16-bit weights,
                            the tiled receive, delay >= 3): the update of step t and the receive of
                            step t, which delivers S_{t-d+1}, touch disjoint data once the input is
                            held in two buffers, one per step parity.  Results are the same */

/* snn_config.receive */
#define SNN_RECV_AUTO 0u   /* the library measures: snn_build_graph runs every form that applies to the
                              graph (global; with sorted rows tiled, and tiled fused with the update;
                              for the fixed models without plasticity the persistent launch with the
                              fewest CTAs that cover the update and with every resident CTA --
                              SNN_F_SERIAL leaves the fused and persistent forms out) from the initial
                              state over the same
                              delay + 150 steps (at most 1,100) and times the last 48 with CUDA events;
                              the fastest is kept (snn_info.tune_ms) and the state returns to N_0.  A
                              form whose first 32 steps already took twice the best ms/step so far
                              stops there (tune_ms holds that estimate).
                              Results do not depend on the form.  The bulk form is not a candidate */
#define SNN_RECV_GLOBAL 1u /* a warp per row piece (rows cut into up to 16 pieces when a step has few
                              spikes), red.global.add into L2-resident accumulators */
#define SNN_RECV_TILED 2u  /* target-tiled, accumulators in shared memory; needs sorted rows */
#define SNN_RECV_BULK 3u   /* as TILED, rows staged into shared memory by bulk async copies */
#define SNN_RECV_PERSISTENT 4u /* the fixed models without plasticity: each snn_step call is one cooperative
                                  launch that runs its steps as phases (Update Neurons, then the global
                                  receive) separated by a bounded grid-wide barrier; no launch per kernel */

typedef struct {
    uint32_t model;        /* snn_model */
    uint32_t flags;        /* SNN_F_* */
    uint32_t delay;        /* d >= 1 steps; a spike of step t reaches the update of step t+d */
    uint32_t n_inst;       /* number of network instances, >= 1 */
    uint64_t seed;         /* Philox key word 0 (word 1 is inst_key0 + the instance index) */
    uint64_t log_capacity; /* spikes the raster log keeps (0: no log), shared out
                              among the instances in proportion to their
                              neurons: instance b keeps floor(log_capacity
                              n_b / N) of its spikes; one that fills its share
                              sets SNN_E_OVERFLOW */
    uint32_t receive;      /* SNN_RECV_* */
    uint32_t steps_per_graph; /* steps captured per CUDA graph (0: library default) */
    uint32_t tune_steps;   /* bulk-copy receive: at this step and at 8x this step of the
                              first run its static work items are re-cut by the spike
                              counts measured since the previous cut (0: 256, 0xffffffff:
                              never); the tiled receive cuts its items on the device every
                              step.  Results do not depend on the plan */
    uint32_t lazy_fifo;    /* SNN_F_LAZY: steps of spike and trace history kept per neuron, the
                              longest a row stays stale (0: 128, the most the two 64-bit
                              history words of a neuron hold; else 2..128.  The paper's queue
                              holds 50 entries) */
    uint32_t wait_polls;   /* polls of one bounded device-side wait before the kernel gives up with
                              SNN_E_TIMEOUT: a producer or consumer wait on an mbarrier of the bulk-copy
                              receive (0: 2^20; the wait for the copies still in flight before a CTA
                              exits keeps its own bound of 2^26 polls), or a grid-barrier wait of the
                              persistent launch (0: 2^22 polls, 64 ns apart) */
    uint32_t inst_key0;    /* Philox key word 1 of instance 0: instance b draws with key (seed,
                              inst_key0 + b), so that one network of a batch re-run alone in its
                              own context gets the same random numbers (0 for a batch) */
} snn_config;

/* Model constants of one instance.  Times in ms, potentials in mV, integer
 * weights in lattice units (2^-16 mV).  Every binary32 constant the update
 * uses is the binary64 expression below rounded once to nearest. */
typedef struct {
    uint32_t n;                /* neurons of this instance (local ids 0..n-1) */
    uint32_t n_exc;            /* local ids < n_exc are excitatory */
    uint32_t refractory_steps; /* R <= 255: steps clamped at v_reset after a spike */
    int32_t jext_q;            /* Brunel: lattice units per external Poisson spike */
    int32_t w_max_q;           /* STDP: plastic weights are clipped to [0, w_max_q] */
    uint32_t reserved;
    double dt, tau_m;          /* Pm = exp(-dt/tau_m) */
    double v_th, v_reset;
    double e_l, tau_e, tau_i;  /* Vogels: resting drive, Pe = exp(-dt/tau_e), Pi = exp(-dt/tau_i) */
    double lambda;             /* Brunel: Poisson mean of external spikes per step */
    double v0_lo, v0_span;     /* V0 = v0_lo + v0_span * u, u uniform on [0,1) in steps of 2^-24 */
    double tau_plus, tau_minus;/* STDP trace time constants */
    double a_plus, a_minus;    /* STDP amplitudes as fractions of w_max_q */
} snn_params;

/* Device memory and stream.  alloc/free may be NULL (then cudaMalloc and
 * cudaFree are used).  stream is a cudaStream_t (NULL: the legacy default
 * stream).  The library calls alloc/free inside snn_create,
 * snn_build_graph and snn_destroy, for temporary buffers inside
 * snn_read_spikes, snn_read_state / snn_write_state of SNN_FIELD_W and
 * snn_stats, and (SNN_RECV_BULK only) inside snn_step at the two re-plans
 * of its work items; snn_rate_cv_static allocates nothing.  Large host copies go
 * through a pinned staging ring of 256 MB that the context allocates at
 * the first one and frees in snn_destroy. */
typedef struct {
    void* (*alloc)(size_t bytes, void* stream, void* user);
    void (*free)(void* ptr, void* stream, void* user);
    void* user;
    void* stream;
} snn_device;

/* Create a context for n_inst instances (params is an array of n_inst).
 * The instances are concatenated in order: global neuron id = sum of the
 * sizes of the earlier instances + local id.  Returns SNN_E_ARG for an
 * invalid config (delay 0 or > 1000, refractory > 255, STDP without
 * Brunel, SNN_F_LAZY without SNN_F_STDP or lazy_fifo outside 2..128,
 * non-positive time constants, lambda < 0 or so large that the Poisson
 * table would exceed 64 entries).  *out is NULL on failure. */
snn_status snn_create(const snn_config* cfg, const snn_params* params, const snn_device* dev,
                      snn_ctx** out);

/* Load the graph (host pointers; the library copies them and keeps no
 * reference).  row_off[N+1] are CSR row offsets over global neuron ids
 * (row_off[0] == 0, non-decreasing), tgt[E] the targets of each row, w_q[E]
 * the weights in lattice units.  Targets must lie in the source's instance.
 * With SNN_F_W16 every row must be representable as int16 codes times one
 * power of two, 2^s with s <= 15 (plastic rows with s == 0); without it
 * every weight must satisfy |w| <= 2^24.  Rows need not be sorted; sorted
 * rows give better locality (Section III-A-2).  Violations give SNN_E_ARG
 * and leave no graph loaded.  On success the neuron state is initialised
 * (the paper's Init stage, Fig. 1) and the step counter is 0. */
snn_status snn_build_graph(snn_ctx* ctx, const uint64_t* row_off, const uint32_t* tgt, const int32_t* w_q);

/* snn_build_graph for a graph whose rows each carry one weight, the
 * population-typed synapses of Table 2 (Section III-A-2: the Vogels and
 * Brunel networks store no weight per synapse): w_row[N] is the weight of
 * every synapse of row j, in lattice units.  The result is that of
 * snn_build_graph with w_q[e] = w_row[j] for e in [row_off[j], row_off[j+1]),
 * including what snn_read_state(SNN_FIELD_W) returns, but only the targets
 * and N weights cross the bus.  The caller vouches that the rows are of
 * that form; the same argument checks apply otherwise. */
snn_status snn_build_graph_rows(snn_ctx* ctx, const uint64_t* row_off, const uint32_t* tgt, const int32_t* w_row);

/* (Re)initialise the neuron state N_0 and restore the weights loaded by
 * snn_build_graph; the step counter returns to 0 and the log is cleared. */
snn_status snn_reset(snn_ctx* ctx);

/* Enqueue n_steps timesteps on the context's stream and return without
 * waiting.  Device-side errors surface at the next call that synchronises.
 * With the bulk-copy receive, a call that crosses a re-plan step (see
 * cfg.tune_steps; twice per graph load) waits for the device, re-cuts the
 * work items by the measured work and re-captures its CUDA graphs before
 * going on. */
snn_status snn_step(snn_ctx* ctx, uint32_t n_steps);

/* Run n_steps timesteps without the CUDA graph, with CUDA events around
 * every kernel of the step, and wait for them.  phase_ms[6] receives the
 * summed device time of each phase: [0] Update Synapses (depression),
 * [1] Update Neurons, [2] Update Synapses (potentiation), [3] Receive
 * Spikes (the receive kernel; with the tiled receive also any wait for its
 * per-step plan, which runs beside [0]-[2] when the delay is 2 or more and
 * before [3] otherwise; with the fused step the one kernel that runs Update
 * Neurons and Receive Spikes together, [1] then 0), [4] the merge of the receive's partial
 * accumulators, [5] end-of-step bookkeeping.  Used to measure one kernel's
 * share of the step; the simulation advances exactly as with snn_step. */
snn_status snn_step_profiled(snn_ctx* ctx, uint32_t n_steps, double* phase_ms);

/* Wait for the enqueued work; returns the first pending device-side error. */
snn_status snn_sync(snn_ctx* ctx);

/* Spikes of steps [t0, t1) from the raster log, sorted by (step, global
 * id), written to steps[] and ids[] (each of capacity cap).  *n_out gets the
 * number of such spikes; with cap == 0 only the count is returned, with
 * cap < count SNN_E_OVERFLOW is returned and nothing is written.  If an
 * instance filled its share of the log, *n_out counts the spikes kept and
 * SNN_E_OVERFLOW is returned.  Synchronises. */
snn_status snn_read_spikes(snn_ctx* ctx, uint32_t t0, uint32_t t1, uint32_t* steps, uint32_t* ids,
                           uint64_t cap, uint64_t* n_out);

/* Drop the logged spikes; logging continues from the current step. */
snn_status snn_log_clear(snn_ctx* ctx);

/* State fields for snn_read_state / snn_write_state (N entries in global
 * id order unless noted). */
typedef enum {
    SNN_FIELD_V = 0,    /* float, mV */
    SNN_FIELD_GE = 1,   /* float, mV (Vogels) */
    SNN_FIELD_GI = 2,   /* float, mV (Vogels) */
    SNN_FIELD_R = 3,    /* int32, refractory steps left */
    SNN_FIELD_X = 4,    /* float, presynaptic STDP trace */
    SNN_FIELD_Y = 5,    /* float, postsynaptic STDP trace */
    SNN_FIELD_ACC0 = 6, /* int32, pending input (channel 0: excitatory / all) */
    SNN_FIELD_ACC1 = 7, /* int32, pending input (channel 1: Vogels inhibitory) */
    SNN_FIELD_W = 8,    /* int32[E], weights in lattice units, CSR order of snn_build_graph */
    SNN_FIELD_MODEL = 9 /* generic models: N records of snn_info.model_state_bytes bytes each, the
                           model's neuron struct (SNN_MODEL_RELAY: uint8 flag; SNN_MODEL_BRUNEL_LIF:
                           float V, uint8 refractory steps left, 3 bytes padding) */
} snn_field;

/* Copy a state field to / from host memory (synchronises).  Writing takes
 * effect before the next step; it is how tests force a spike.  The queues
 * of the delay FIFO are not part of these fields.  With SNN_F_LAZY, reading
 * or writing W or X first brings every stale row up to date (a pass over
 * the plastic rows; the values are those of the eager rule). */
snn_status snn_read_state(snn_ctx* ctx, snn_field field, void* host);
snn_status snn_write_state(snn_ctx* ctx, snn_field field, const void* host);

/* Counters since the last reset: steps done, spikes emitted and synaptic
 * events delivered (sum of the row lengths of the delivered spikes). */
snn_status snn_counters(snn_ctx* ctx, uint64_t* steps, uint64_t* spikes, uint64_t* events);

/* Population rate (Hz) of one instance since the statistics window began
 * (step 0 or the last snn_stats_clear), and the mean ISI coefficient of
 * variation over its neurons with at least 3 spikes in the window (needs
 * SNN_F_STATS; reductions in binary64 on the device). */
snn_status snn_stats(snn_ctx* ctx, uint32_t inst, double* rate_hz, double* isi_cv);

/* Start the statistics window at the current step. */
snn_status snn_stats_clear(snn_ctx* ctx);

/* Population rate and mean ISI CV computed without allocating any device
 * memory.  The paper has no counterpart; this exists for callers that cannot
 * call cudaMalloc when they want the numbers: applications that give the
 * GPU's memory to their own fixed arena at start-up, and latency-critical
 * loops where an allocation may synchronise the device.
 *
 * Inputs are device arrays of n neurons: count[i] spikes in the window,
 * isi_sum[i] and isi_sq[i] the sum and the sum of squares of the neuron's
 * inter-spike intervals in steps (the layout snn_stats keeps internally).
 * window_steps * dt_ms is the window length.  Results go to *rate_hz and
 * *isi_cv (host), with the same definitions as snn_stats; the partial sums
 * are added in a fixed order, so repeated calls give identical results.
 * Work is enqueued on `stream` (a cudaStream_t, NULL for the legacy default
 * stream) and the call waits for it.
 *
 * Scratch: a static device array of 8192 * 3 + 3 doubles (192 KB) inside
 * the library, held by every GPU that loads the library until exit, so n is
 * limited to 16,777,216; larger n returns SNN_E_ARG.  The first call on a
 * device looks the array's address up (cudaGetSymbolAddress) and keeps it for
 * the device's current CUDA context; the first call after a cudaDeviceReset
 * looks it up again.  Make the first call on a device before any stream
 * capture begins.  All calls share the array: calls
 * that overlap on the GPU (other streams, other host threads) race and must
 * be serialised by the caller. */
snn_status snn_rate_cv_static(const uint32_t* count, const unsigned long long* isi_sum,
                              const unsigned long long* isi_sq, uint32_t n, uint64_t window_steps, double dt_ms,
                              void* stream, double* rate_hz, double* isi_cv);

/* A job of the adjacency construction (Section III-A-2, Fig. 2): n sorted,
 * unique, uniformly distributed random integers from [a, b), written at
 * out[o .. o + n). */
typedef struct {
    uint32_t n, a, b, reserved;
    uint64_t o;
} snn_job;

/* Expand n_jobs jobs on the GPU (no context needed).  Job j draws its n + 1
 * exponential spacings from Philox4x64-10 with key (seed, j) and counter
 * (k >> 3, 0, 2, 0), word k & 7; value k = 1..n is a + round(c_k / c_{n+1}
 * (b - a - n)) + (k - 1), c_k the exclusive running sum of the spacings.
 * jobs and out are device pointers (out_len elements); stream is a CUDA
 * stream (NULL: the legacy default stream).  Waits for the stream.  Errors:
 * SNN_E_ARG for n_jobs >= 2^32 or a job with b < a, n > b - a,
 * b - a - n > 2^24 or o + n > out_len (that job writes nothing; the others
 * are written); SNN_E_CUDA.  Allocates nothing: the invalid-job flag is one
 * static device word that every call clears and reads, so calls that
 * overlap on the GPU (other streams, other host threads) race on it and must
 * be serialised by the caller. */
snn_status snn_expand_jobs(const snn_job* jobs, uint64_t n_jobs, uint64_t seed, uint32_t* out, uint64_t out_len,
                           void* stream);

/* What the context chose and holds. */
typedef struct {
    uint32_t receive;      /* the receive form in use: SNN_RECV_GLOBAL, _TILED or _BULK (after snn_build_graph) */
    uint32_t n_tiles;      /* target tiles of the tiled receive (0: global) */
    uint32_t n_padded;     /* neuron slots on the device (instances padded to 256) */
    uint32_t rows_sorted;  /* 1 if every row's targets ascend */
    uint64_t edges;        /* synapses loaded */
    uint64_t device_bytes; /* device memory held */
    uint32_t edge_bytes;   /* bytes the receive reads per delivered edge: 4 (packed edges, or targets alone
                              with row weights), 6 (u32 targets + int16 codes), 8 (+ binary32 weights) */
    uint32_t model_state_bytes; /* generic models: bytes of one neuron's state record (else 0) */
    uint32_t fused;        /* 1: update and receive of a step run in one kernel (see SNN_F_SERIAL) */
    uint32_t tuned;        /* 1: the receive form was chosen by SNN_RECV_AUTO's timing run */
    float tune_ms[5];      /* SNN_RECV_AUTO: ms per step each form took in that run, in the order global,
                              tiled (separate kernels), tiled fused with the update, bulk, persistent
                              launch (the better of its two grids); 0: not a candidate for this graph */
    uint32_t persistent;   /* 1: one cooperative launch per snn_step call (SNN_RECV_PERSISTENT) */
    uint32_t persist_ctas; /* its CTAs of 256 threads */
} snn_info;
snn_status snn_get_info(snn_ctx* ctx, snn_info* info);

const char* snn_last_error(const snn_ctx* ctx); /* never NULL; ctx may be NULL */
const char* snn_status_string(snn_status s);
void snn_destroy(snn_ctx* ctx); /* NULL-safe */

#ifdef __cplusplus
}
#endif
#endif
