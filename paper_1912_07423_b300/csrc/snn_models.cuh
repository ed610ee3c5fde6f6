// snn_models.cuh -- the generic update of libsnn (Section III-B): neuron
// models written as device functors with init() and update() callbacks,
// compiled into the library and selected by snn_config.model.
//
// A model is a struct with
//   struct neuron { ... };            per-neuron state, trivially copyable (one
//                                     record per neuron, SNN_FIELD_MODEL)
//   static constexpr bool kRandom;    whether update() wants a random word
//   __device__ static void init(neuron&, const ModelView&, uint32_t local, uint32_t word);
//   __device__ static bool update(neuron&, const ModelView&, int32_t input, uint32_t word);
// init() runs once per neuron (word: the Philox word of tag 0 at step 0);
// update() runs once per neuron and step and returns whether it spikes
// (word: the Philox word of tag 1 at that step, input: the sum of the
// lattice weights the neuron received since its last update).  The paper's
// receive() callback is the library's Receive Spikes: integer sums, whose
// order does not matter, so every model stays deterministic.  Spikes go to
// the work queue, the delay FIFO and the raster log exactly as for the
// fixed models.  Building blocks compose by inheritance (Fig. 5d: Brunel
// from the LIF block).
#pragma once
#include "snn_kernels.cuh"
#include "../../include/snn.h"

namespace snn {

// What a model's callbacks see of its instance.
struct ModelView {
    const InstDev* I;    // the instance's constants (binary32, see InstDev)
    const uint32_t* T;   // Poisson thresholds
    const uint8_t* S;    // Poisson bucket table
    uint32_t nT;
    // external Poisson drive: spikes of this step for a uniform 32-bit word
    __device__ __forceinline__ uint32_t poisson(uint32_t u) const { return poisson_count(T, S, nT, u); }
};

// Leaky integrate-and-fire building block: V relative to rest, V <- V Pm +
// input, threshold v_th, reset to v_reset, R clamped steps during which
// input is discarded.
struct LifBlock {
    struct neuron {
        float V;
        uint8_t r;
    };
    // V0 = v0_lo + v0_span u, u uniform on [0, 1) in steps of 2^-24
    __device__ static void init(neuron& s, const ModelView& m, uint32_t, uint32_t word)
    {
        const float u01 = __fmul_rn(__uint2float_rn(word >> 8), 1.0f / 16777216.0f);
        s.V = __fadd_rn(m.I->v0_lo, __fmul_rn(m.I->v0_span, u01));
        s.r = 0;
    }
    __device__ static bool refractory(const neuron& s) { return s.r > 0; }
    // one step with input in mV
    __device__ static bool step(neuron& s, const ModelView& m, float in)
    {
        if (s.r > 0) {
            s.r = (uint8_t)(s.r - 1);
            s.V = m.I->v_reset;
            return false;
        }
        s.V = __fadd_rn(__fmul_rn(s.V, m.I->Pm), in);
        if (s.V >= m.I->v_th) {
            s.V = m.I->v_reset;
            s.r = (uint8_t)m.I->R;
            return true;
        }
        return false;
    }
};

// Brunel (Section IV) from the LIF block: the block's update specialised
// with the external Poisson drive (drawn only outside the refractory
// clamp, whose input is discarded).
struct BrunelLif : LifBlock {
    static constexpr bool kRandom = true;
    __device__ static bool update(neuron& s, const ModelView& m, int32_t input, uint32_t word)
    {
        if (refractory(s)) return step(s, m, 0.0f);
        const int32_t in = input + (int32_t)m.poisson(word) * m.I->jext;
        return step(s, m, __fmul_rn(__int2float_rn(in), kLattice));
    }
};

// The paper's tutorial model (Listing 1): a neuron holds one flag; the
// first population (local ids < n_exc) starts set; a neuron fires when its
// flag is set or it received input since its last update, and clears the
// flag, so that activity hops from population to population.
struct RelayModel {
    struct neuron {
        uint8_t flag;
    };
    static constexpr bool kRandom = false;
    __device__ static void init(neuron& s, const ModelView& m, uint32_t local, uint32_t)
    {
        s.flag = local < m.I->n_exc ? 1 : 0;
    }
    __device__ static bool update(neuron& s, const ModelView&, int32_t input, uint32_t)
    {
        const bool fire = s.flag != 0 || input != 0;
        s.flag = 0;
        return fire;
    }
};

// K consecutive records to or from registers, with 16- or 8-byte accesses
// where the K records fill them (the array is 256-byte aligned and starts
// at a multiple of K records).
template <class T, int K>
__device__ __forceinline__ void copy_records(T* __restrict__ dst, const T* __restrict__ src)
{
    constexpr size_t bytes = sizeof(T) * K;
    if constexpr (bytes % 16 == 0) {
#pragma unroll
        for (size_t h = 0; h < bytes / 16; ++h) reinterpret_cast<uint4*>(dst)[h] = reinterpret_cast<const uint4*>(src)[h];
    } else if constexpr (bytes % 8 == 0) {
#pragma unroll
        for (size_t h = 0; h < bytes / 8; ++h) reinterpret_cast<uint2*>(dst)[h] = reinterpret_cast<const uint2*>(src)[h];
    } else {
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = src[k];
    }
}

__device__ __forceinline__ ModelView model_view(const Net& n, uint32_t b)
{
    ModelView v;
    v.I = n.inst + b;
    v.T = n.pois + __ldg(&v.I->pois_off);
    v.S = n.pois_start + (size_t)b * kPoissonBuckets;
    v.nT = __ldg(&v.I->pois_n);
    return v;
}

// Init stage for a generic model: init() of every neuron.
template <class M>
__global__ void k_init_model(Net n, typename M::neuron* __restrict__ ms)
{
    constexpr int K = 8;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n.Np / K) return;
    const uint32_t id0 = g * K;
    const uint32_t b = n.inst_of_w32[id0 >> 5];
    const ModelView mv = model_view(n, b);
    const uint32_t local0 = id0 - mv.I->pbase;
    uint32_t words[8];
    philox_words8(n.seed, n.key0 + b, local0 >> 3, 0, 0, words);
    alignas(16) typename M::neuron st[K];
    for (int k = 0; k < K; ++k) {
        st[k] = typename M::neuron{};
        if (local0 + k < mv.I->n) M::init(st[k], mv, local0 + k, words[k]);
    }
    copy_records<typename M::neuron, K>(ms + id0, st);
}

// Update Neurons for a generic model: the same work queue, delay FIFO,
// raster log and statistics as k_update, with the model's update() in the
// place of the fixed equations.
template <class M, bool STATS>
__global__ void __launch_bounds__(256) k_update_model(Net n, typename M::neuron* __restrict__ ms)
{
    constexpr int NPT = kUpdateNeurons;
    const unsigned long long t = n.ctl->t + n.k;
    step_bookkeeping(n, t, blockIdx.x * blockDim.x + threadIdx.x, false);  // of the previous step, as in k_update
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const uint32_t G = n.Np / NPT;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = g < G;
    const uint32_t id0 = g * NPT;
    uint32_t spk = 0;
    alignas(16) typename M::neuron st[NPT];
    int32_t a0[NPT];
    if (active) {
        copy_records<typename M::neuron, NPT>(st, ms + id0);
#pragma unroll
        for (int h = 0; h < NPT / 4; ++h)
            *reinterpret_cast<int4*>(a0 + 4 * h) = *reinterpret_cast<const int4*>(n.acc0 + id0 + 4 * h);
    }
    const uint32_t b = active ? __ldg(n.inst_of_w32 + (id0 >> 5)) : 0u;
    const ModelView mv = model_view(n, b);
    const uint32_t pbase = active ? __ldg(&mv.I->pbase) : 0u;
    if (active) {
        const uint32_t nloc = __ldg(&mv.I->n);
        const uint32_t local0 = id0 - pbase;
        if (local0 < nloc) {
            uint32_t words[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if (M::kRandom) philox_words8(n.seed, n.key0 + b, local0 >> 3, t, 1, words);
#pragma unroll
            for (int k = 0; k < NPT; ++k) {
                if (local0 + k >= nloc) continue;
                if (M::update(st[k], mv, a0[k], words[k])) spk |= 1u << k;
            }
            copy_records<typename M::neuron, NPT>(ms + id0, st);
#pragma unroll
            for (int h = 0; h < NPT / 4; ++h) *reinterpret_cast<int4*>(n.acc0 + id0 + 4 * h) = make_int4(0, 0, 0, 0);
            if (STATS && spk) {
#pragma unroll
                for (int k = 0; k < NPT; ++k)
                    if (spk >> k & 1u) {
                        const uint32_t c = n.st_cnt[id0 + k];
                        if (c > 0) {
                            const unsigned long long isi = t - n.st_last[id0 + k];
                            n.st_sum[id0 + k] += isi;
                            n.st_sq[id0 + k] += isi * isi;
                        }
                        n.st_cnt[id0 + k] = c + 1;
                        n.st_last[id0 + k] = (uint32_t)t;
                    }
            }
        }
    }

    // spike compaction into the instance's queue region and the raster log,
    // as in k_update
    const uint32_t lane = lane_id();
    const uint32_t slot_q = (uint32_t)(t % n.D);
    const uint32_t slot_c = (uint32_t)(t & (n.cr - 1));
    const uint32_t c = __popc(spk);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total == 0) return;
    uint32_t wbase = 0;
    if (lane == 31) wbase = atomicAdd(&n.icount[(size_t)slot_c * n.n_inst + b], total);
    const LogSlot L = spk ? log_slot(n, t, b) : LogSlot{0ull, 0ull, 0ull};
    wbase = __shfl_sync(kFull, wbase, 31);
    if (spk) file_spikes(n, t, id0, spk, incl - c, slot_q, pbase, wbase, L);
}

// ---------------------------------------------------------------------------
// Host-side dispatch over the compiled models.
// ---------------------------------------------------------------------------
inline bool is_generic_model(uint32_t model) { return model == SNN_MODEL_RELAY || model == SNN_MODEL_BRUNEL_LIF; }

inline size_t model_state_bytes(uint32_t model)
{
    switch (model) {
    case SNN_MODEL_RELAY: return sizeof(RelayModel::neuron);
    case SNN_MODEL_BRUNEL_LIF: return sizeof(BrunelLif::neuron);
    default: return 0;
    }
}

template <class M>
inline void launch_update_model_t(const Net& n, void* ms, bool stats, uint32_t blocks, cudaStream_t s)
{
    auto* p = static_cast<typename M::neuron*>(ms);
    if (stats)
        k_update_model<M, true><<<blocks, 256, 0, s>>>(n, p);
    else
        k_update_model<M, false><<<blocks, 256, 0, s>>>(n, p);
}

inline void launch_update_model(uint32_t model, const Net& n, void* ms, bool stats, uint32_t blocks, cudaStream_t s)
{
    if (model == SNN_MODEL_RELAY) launch_update_model_t<RelayModel>(n, ms, stats, blocks, s);
    if (model == SNN_MODEL_BRUNEL_LIF) launch_update_model_t<BrunelLif>(n, ms, stats, blocks, s);
}

inline void launch_init_model(uint32_t model, const Net& n, void* ms, uint32_t blocks, cudaStream_t s)
{
    if (model == SNN_MODEL_RELAY) k_init_model<RelayModel><<<blocks, 256, 0, s>>>(n, static_cast<RelayModel::neuron*>(ms));
    if (model == SNN_MODEL_BRUNEL_LIF)
        k_init_model<BrunelLif><<<blocks, 256, 0, s>>>(n, static_cast<BrunelLif::neuron*>(ms));
}

}  // namespace snn
