// snn_device.cuh -- device-side data layout and helpers of libsnn.
//
// Layout in HBM (structure of arrays, Section III-A-2):
//   neurons  : instance b occupies padded ids [pbase_b, pbase_b + n_b) with
//              pbase_b a multiple of 256, so the 256 neurons one warp of the
//              update kernel advances (8 per thread) never straddle two
//              instances.
//              V, ge, gi, x, y: float[Np]; r: uint8[Np]; acc0, acc1: int32[Np];
//              with the fused step a second channel-0 buffer accx: int32[Np]
//              (the input of step t is in acc0 for even t, accx for odd t).
//   graph    : CSR over padded ids, roff: uint64[Np+1], tgt: uint32[E]
//              (padded ids, sorted rows), weights int16[E] (code, value =
//              code << shift(row)) or float[E] (exact lattice integers),
//              meta: uint8[Np] = shift | exc_source << 6 | channel << 7;
//              when every row carries one weight (the source population's),
//              roww: int32[Np] holds it and the global receive reads the
//              targets alone.
//   queues   : the delay FIFO is a ring of D spike queues, uint32[D][Np]
//              (Section III-A-2: arrays with an atomic insertion index).  In
//              every slot instance b owns the region [pbase_b, pbase_b+n_b)
//              with its own index icount[t % CR][b], so a consumer can take
//              one network's spikes alone.  With STDP a ring of D spike
//              bitmasks uint32[D][Np/32] sits beside it (Section III-A-1).
//   log      : the raster log, (step << 32 | padded id) per spike; instance b
//              appends to its own region [log_lo_b, log_lo_b + log_n_b) in
//              step order, a warp's spikes at the instance's logged count
//              before the step plus the warp's queue position, so filing a
//              spike takes the one queue-index atomic and no step-wide one.
//   lazy     : lazy Update Synapses (Section III-A-1): per neuron a 128-bit
//              spike history hist[2 Np] (bit k: spiked at step t - k; words
//              2i and 2i+1 hold bits 0..63 and 64..127 of neuron i), a ring
//              of F decayed postsynaptic traces yring[F][Np] (slot s % F:
//              y(s-1) P-, the value a depression at step s reads), the
//              row's age[Np] (first step whose synaptic events the row has
//              not seen, 31 bits, | an arrival-pending flag << 31), and the
//              queue xq[Np] of rows whose age reaches F this step.
#pragma once
#include <cstdint>

namespace snn {

constexpr int kPad = 256;         // instance alignment in neurons
constexpr int kPoissonCap = 64;   // Poisson threshold table entries per instance
constexpr int kPoissonBuckets = 256;  // buckets of the top 8 bits of a draw
constexpr float kLattice = 1.0f / 65536.0f;  // 2^-16 mV

enum : uint32_t {
    kErrLogOverflow = 1u,
    kErrBadTarget = 2u,
    kErrBadWeight = 4u,
    kErrPlasticShift = 8u,
    kErrTimeout = 16u,
    kErrPlan = 32u,  // the per-step receive plan did not fit its buffer (not reached: the buffer is sized for the bound)
    kErrLazyAge = 64u,  // a lazy row was older than its history (not reached: expiring rows are replayed in time)
};

// Per-instance constants, each binary32 value the binary64 expression
// rounded once (see snn_params in snn.h).
struct InstDev {
    uint32_t pbase, n, n_exc, R;
    uint32_t goff, pad;  // first global neuron id of the instance
    int32_t jext, wmax;
    uint32_t pois_off, pois_n;
    float Pm, Pe, Pi, Pp, Pn, Ap, Am;
    float v_th, v_reset, e_l, v0_lo, v0_span;
    unsigned long long log_lo, log_n;  // the instance's region of the raster log: first entry, entries
};

// Device control block: the step counter and the work-queue indices.
struct Ctl {
    unsigned long long t;       // current step
    unsigned long long t_log0;  // first step of the raster log
    unsigned long long t_stat0; // first step of the statistics window
    unsigned long long events;  // delivered synaptic events
    unsigned long long spikes;  // emitted spikes
    unsigned int err;           // kErr* bits
    unsigned int pad;
};

// Everything a kernel needs, passed by value.
struct Net {
    uint32_t Np, D, d, n_inst;
    uint32_t cr;               // count-ring length, a power of two >= D + 2
    uint32_t k;                // this launch's step offset: step = ctl->t + k
    uint32_t F;                // lazy plasticity: history length in steps (2..128)
    uint32_t key0;             // Philox key word 1 of instance 0 (instance b uses key0 + b)
    uint32_t pad0;
    uint64_t seed;
    unsigned int* icount;      // |S_t| of instance b at [(t % cr) * n_inst + b]
    unsigned long long* ilog;  // spikes of instance b logged before step t, at [(t & 1) * n_inst + b]
    unsigned long long* inst_spikes; // spikes of each instance since the last reset
    unsigned int* tile_ctr;    // tiled receive: next tile to take, at [t & 1]
    const InstDev* inst;
    const uint32_t* inst_of_w32;  // instance of each 32-neuron word
    const uint4* wdesc;           // per 32-neuron word: instance, its pbase, its n (the update's first load)
    const uint32_t* pois;         // Poisson thresholds, kPoissonCap per instance
    const uint8_t* pois_start;    // per instance kPoissonBuckets counts: thresholds < h 2^24
    float* V;
    float* ge;
    float* gi;
    float* x;
    float* y;
    uint8_t* r;
    int32_t* acc0;
    int32_t* acc1;
    int32_t* accx;          // fused step: the second channel-0 input buffer (the update of step t
                            // reads buffer t & 1: acc0 for even t, accx for odd t)
    const uint64_t* roff;
    const uint32_t* tgt;
    int16_t* w16;
    float* w32;
    const uint8_t* meta;
    const uint4* rinfo;     // per padded row: start (lo, hi), length, meta -- one load per spike
    const int32_t* roww;    // row weights (lattice units) when every row carries one (null otherwise)
    const uint32_t* pk;     // packed edges for the tiled receive (null when not used)
    const uint16_t* pk16;   // 16-bit target offsets for the tiled receive with row weights (null when not used)
    const uint64_t* coff;   // STDP: plastic in-edges per padded post id
    const uint32_t* cedge;  // STDP: edge index of each plastic in-edge
    const uint32_t* cpre;   // STDP: padded presynaptic id of each plastic in-edge
    uint32_t* q;            // D * Np
    uint32_t* bits;         // D * Np/32
    unsigned long long* hist;  // lazy: 2 words of spike history per neuron, bit k = step t - k
    float* yring;           // lazy: F * Np decayed postsynaptic traces
    uint32_t* age;          // lazy: per row, first step not applied | arrival pending << 31
    uint32_t* xq;           // lazy: rows whose history expires at this step
    unsigned int* xcount;   // lazy: entries of xq, at [t & 1]
    unsigned long long* log;
    unsigned long long log_cap;
    uint32_t* st_cnt;
    uint32_t* st_last;
    unsigned long long* st_sum;
    unsigned long long* st_sq;
    Ctl* ctl;
};

// ---------------------------------------------------------------------------
// Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11), written from its
// published definition: 10 rounds of two 64x64->128 multiplications with a
// Weyl-sequence key schedule.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(uint64_t& c0, uint64_t& c1, uint64_t& c2, uint64_t& c3, uint64_t k0,
                                              uint64_t k1)
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
#pragma unroll
    for (int round = 0; round < 10; ++round) {
        if (round) {
            k0 += W0;
            k1 += W1;
        }
        const uint64_t hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const uint64_t hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const uint64_t n0 = hi1 ^ c1 ^ k0;
        const uint64_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
    }
}

// The 8 words of the block at counter (group, step, tag, 0), key (seed,
// instance): word k belongs to local neuron 8*group + k, low half first.
__device__ __forceinline__ void philox_words8(uint64_t seed, uint32_t inst, uint32_t group, uint64_t step,
                                              uint32_t tag, uint32_t w[8])
{
    uint64_t c0 = group, c1 = step, c2 = tag, c3 = 0;
    philox4x64_10(c0, c1, c2, c3, seed, inst);
    w[0] = (uint32_t)c0; w[1] = (uint32_t)(c0 >> 32);
    w[2] = (uint32_t)c1; w[3] = (uint32_t)(c1 >> 32);
    w[4] = (uint32_t)c2; w[5] = (uint32_t)(c2 >> 32);
    w[6] = (uint32_t)c3; w[7] = (uint32_t)(c3 >> 32);
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }

}  // namespace snn
