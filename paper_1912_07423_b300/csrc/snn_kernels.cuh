// snn_kernels.cuh -- the per-step kernels of libsnn (Update Neurons with
// spike compaction, Update Synapses in its eager and lazy forms, the
// global-atomic Receive Spikes) and the set-up kernels.  The tiled and
// bulk-copy receives are in snn_tiled.cuh and snn_bulk.cuh, the generic
// update in snn_models.cuh.
//
// Arithmetic of the neuron update: binary32, one rounding per operation, no
// contraction (explicit __f*_rn intrinsics; the file is also compiled with
// -fmad=false), in the order documented in snn.h / the oracle's header.
#pragma once
#include <cuda_runtime.h>

#include "snn_device.cuh"

namespace snn {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Update Neurons (Section III-A-1): N_t -> N'_{t+1}, spikers -> S_t.
// One thread advances NPT consecutive neurons (8, or 4 where 8 would leave
// SMs idle or take too many registers; 128-bit loads per float field) and
// computes one Philox block, whose 8 words are the Poisson draws of an
// aligned group of 8 neurons.  Spiking ids are compacted per warp with a
// shuffle scan and one atomicAdd on the queue index (Section III-A-2:
// queues are arrays with an atomic index).
// ---------------------------------------------------------------------------

constexpr int kUpdateNeurons = 8;       // neurons per thread of the update
constexpr int kUpdateNeuronsSmall = 4;  // ... when 8 per thread would leave SMs without a block
// a warp of the update covers 32 * NPT neurons and must never cross an
// instance (instances are padded to 256 slots): its spikes go to one
// instance's queue region with one atomicAdd
static_assert(256 % (32 * kUpdateNeurons) == 0, "a warp of the update must stay inside one 256-slot block");
static_assert(256 % (32 * kUpdateNeuronsSmall) == 0, "a warp of the update must stay inside one 256-slot block");

// Number of Poisson thresholds <= u (thresholds T[0..nT) ascending): the
// instance's bucket table S gives the count below the start of u's bucket
// (S[h] = thresholds < h 2^24), and the thresholds inside the bucket are
// passed one by one -- usually none or one.
__device__ __forceinline__ uint32_t poisson_count(const uint32_t* __restrict__ T, const uint8_t* __restrict__ S,
                                                  uint32_t nT, uint32_t u)
{
    uint32_t k = __ldg(S + (u >> 24));
    while (k < nT && __ldg(T + k) <= u) ++k;
    return k;
}

// Spikes of instance b logged before step t (its raster-log entries of steps
// [t_log0, t)): the count the bookkeeping of step t-1 kept plus the queue
// index of step t-1.  Both are final before step t's update starts, so every
// warp of that update reads the same value while the bookkeeping of step t
// stores it in the other parity for step t+1.
__device__ __forceinline__ unsigned long long log_base(const Net& n, unsigned long long t, uint32_t b)
{
    if (t <= n.ctl->t_log0) return 0ull;
    return n.ilog[(size_t)((t - 1) & 1ull) * n.n_inst + b] + n.icount[(size_t)((t - 1) & (n.cr - 1)) * n.n_inst + b];
}

// poisson_count on tables in shared memory.
__device__ __forceinline__ uint32_t poisson_count_s(const uint32_t* T, const uint8_t* S, uint32_t nT, uint32_t u)
{
    uint32_t k = S[u >> 24];
    while (k < nT && T[k] <= u) ++k;
    return k;
}

// Per-step bookkeeping of the previous step, done once per step by the
// threads gt (grid-wide index) of the step's update (its kernels have
// finished): fold its queue indices into the counters, clear the next step's
// indices and the tile counter of the next receive, and keep each instance's
// logged count for the next step.
__device__ __forceinline__ void step_bookkeeping(const Net& n, unsigned long long t, uint32_t gt, bool lazy)
{
    const uint32_t sn = (uint32_t)((t + 1) & (n.cr - 1));
    if (gt < n.n_inst) {
        if (t > 0) {
            const unsigned int c = n.icount[(size_t)((t - 1) & (n.cr - 1)) * n.n_inst + gt];
            n.inst_spikes[gt] += c;
            if (c) atomicAdd(&n.ctl->spikes, (unsigned long long)c);
        }
        n.icount[(size_t)sn * n.n_inst + gt] = 0;
        if (n.log_cap) n.ilog[(size_t)(t & 1ull) * n.n_inst + gt] = log_base(n, t, gt);
    }
    if (gt == 0) {
        n.tile_ctr[(t + 1) & 1ull] = 0;
        if (lazy) n.xcount[(t + 1) & 1ull] = 0;
    }
}

// Where a warp's spikes of step t go in the raster log: its instance's
// logged count before the step (lb) and the instance's log region (lo, cap).
// Loaded while the warp's queue-index atomic is in flight.
struct LogSlot {
    unsigned long long lb, lo, cap;
};

__device__ __forceinline__ LogSlot log_slot(const Net& n, unsigned long long t, uint32_t b)
{
    LogSlot s{0ull, 0ull, 0ull};
    if (n.log_cap) {
        s.lb = log_base(n, t, b);
        s.lo = __ldg(&n.inst[b].log_lo);
        s.cap = __ldg(&n.inst[b].log_n);
    }
    return s;
}

// A warp's spikes into the queue and the raster log: the lane's spikes (bit
// k of spk: neuron id0 + k) at offset off of the warp's range, which starts
// at wbase in instance b's region of queue slot slot_q and at the same place
// after the instance's logged spikes in its log region.
__device__ __forceinline__ void file_spikes(const Net& n, unsigned long long t, uint32_t id0, uint32_t spk, uint32_t off,
                                            uint32_t slot_q, uint32_t pbase, uint32_t wbase, const LogSlot& L)
{
    uint32_t* q = n.q + (size_t)slot_q * n.Np + pbase + wbase + off;
    const unsigned long long lp = L.lb + wbase + off;
    uint32_t m = spk, k = 0;
    while (m) {
        const int bit = __ffs(m) - 1;
        m &= m - 1;
        const uint32_t id = id0 + bit;
        q[k] = id;
        if (n.log_cap) {
            if (lp + k < L.cap)
                n.log[L.lo + lp + k] = (t << 32) | id;
            else
                atomicOr(&n.ctl->err, kErrLogOverflow);
        }
        ++k;
    }
}

// SYN: 0 no plasticity, 1 eager traces (x and y every step), 2 lazy (y, the
// ring of decayed y, the spike history and the expiry queue).  Thread g of
// the step's update advances neurons g*NPT .. g*NPT+NPT-1 (whole warps: a
// warp covers 32*NPT slots inside one instance); acc0 is the channel-0 input
// it reads and clears.
template <int MODEL, int SYN, bool STATS, int NPT, bool SPOIS = false>
__device__ __forceinline__ void update_neurons(const Net& n, unsigned long long t, uint32_t g, int32_t* acc0)
{
    static_assert(NPT == 4 || NPT == 8, "one Philox block serves 8 neurons");
    const uint32_t G = n.Np / NPT;
    const bool active = g < G;  // whole warps: Np is a multiple of 256
    const uint32_t id0 = g * NPT;
    uint32_t spk = 0;  // bit k: neuron id0 + k spiked
    uint32_t xexp = 0;  // lazy plasticity, bit k: the row of id0 + k expires at this step
    bool have = false;  // the group holds neurons (not only padding): its state is stored
    // the state is loaded first: its addresses do not depend on the instance
    // (padding slots are loaded too and left as they are)
    float V[NPT];
    uint8_t r[NPT];
    int32_t a0[NPT];
    if (active) {
#pragma unroll
        for (int h = 0; h < NPT / 4; ++h) {
            *reinterpret_cast<float4*>(V + 4 * h) = *reinterpret_cast<const float4*>(n.V + id0 + 4 * h);
            *reinterpret_cast<uint32_t*>(r + 4 * h) = *reinterpret_cast<const uint32_t*>(n.r + id0 + 4 * h);
            *reinterpret_cast<int4*>(a0 + 4 * h) = *reinterpret_cast<const int4*>(acc0 + id0 + 4 * h);
        }
    }
    // the word's instance, its base and size in one load (uniform across the
    // warp), so the Philox block can start while the instance's constants load
    const uint4 wd = active ? __ldg(n.wdesc + (id0 >> 5)) : make_uint4(0u, 0u, 0u, 0u);
    const uint32_t b = wd.x;
    const InstDev* I = n.inst + b;
    const uint32_t pbase = wd.y;
    // SPOIS (blocks of at most 8 warps): the warp copies its instance's Poisson
    // tables (64 thresholds, 256 bucket counts: 512 bytes) into shared memory
    // while its Philox block is drawn, so the draws' lookups are shared-memory
    // loads (the instance's thresholds sit at pois + kPoissonCap b)
    const uint32_t* Ts = nullptr;
    const uint8_t* Ss = nullptr;
    if constexpr (SPOIS && MODEL == 1) {
        static_assert(kPoissonCap == 64 && kPoissonBuckets == 256, "one 16-byte vector per lane");
        __shared__ uint4 s_pois[8][32];
        const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
        if (active)  // whole warps
            s_pois[warp][lane] = lane < 16 ? __ldg(reinterpret_cast<const uint4*>(n.pois + (size_t)b * kPoissonCap) + lane)
                                           : __ldg(reinterpret_cast<const uint4*>(n.pois_start + (size_t)b * kPoissonBuckets) +
                                                   (lane - 16));
        __syncwarp();
        Ts = reinterpret_cast<const uint32_t*>(&s_pois[warp][0]);
        Ss = reinterpret_cast<const uint8_t*>(&s_pois[warp][16]);
    }

    if (active) {
        const uint32_t nloc = wd.z;
        const uint32_t local0 = id0 - pbase;
        if (local0 < nloc) {
            const float v_th = __ldg(&I->v_th), v_reset = __ldg(&I->v_reset), Pm = __ldg(&I->Pm);
            const uint32_t R = __ldg(&I->R);

            if (MODEL == 0) {  // Vogels-Abbott CUBA
                const float Pe = __ldg(&I->Pe), Pi = __ldg(&I->Pi), e_l = __ldg(&I->e_l);
                float ge[NPT], gi[NPT];
                int32_t a1[NPT];
#pragma unroll
                for (int h = 0; h < NPT / 4; ++h) {
                    *reinterpret_cast<float4*>(ge + 4 * h) = *reinterpret_cast<const float4*>(n.ge + id0 + 4 * h);
                    *reinterpret_cast<float4*>(gi + 4 * h) = *reinterpret_cast<const float4*>(n.gi + id0 + 4 * h);
                    *reinterpret_cast<int4*>(a1 + 4 * h) = *reinterpret_cast<const int4*>(n.acc1 + id0 + 4 * h);
                }
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    if (local0 + k >= nloc) continue;
                    float e = __fadd_rn(ge[k], __fmul_rn(__int2float_rn(a0[k]), kLattice));
                    float i = __fadd_rn(gi[k], __fmul_rn(__int2float_rn(a1[k]), kLattice));
                    float v = V[k];
                    uint32_t rk = r[k];
                    if (rk > 0) {
                        rk -= 1;
                        v = v_reset;
                    } else {
                        const float u = __fadd_rn(e_l, __fadd_rn(e, i));
                        v = __fadd_rn(u, __fmul_rn(__fsub_rn(v, u), Pm));
                    }
                    e = __fmul_rn(e, Pe);
                    i = __fmul_rn(i, Pi);
                    if (rk == 0 && v >= v_th) {
                        spk |= 1u << k;
                        v = v_reset;
                        rk = R;
                    }
                    V[k] = v;
                    ge[k] = e;
                    gi[k] = i;
                    r[k] = (uint8_t)rk;
                }
#pragma unroll
                for (int h = 0; h < NPT / 4; ++h) {
                    *reinterpret_cast<float4*>(n.ge + id0 + 4 * h) = *reinterpret_cast<float4*>(ge + 4 * h);
                    *reinterpret_cast<float4*>(n.gi + id0 + 4 * h) = *reinterpret_cast<float4*>(gi + 4 * h);
                    *reinterpret_cast<int4*>(n.acc1 + id0 + 4 * h) = make_int4(0, 0, 0, 0);
                }
            } else {  // Brunel with Poisson drive
                const int32_t jext = __ldg(&I->jext);
                const uint32_t* T = n.pois + __ldg(&I->pois_off);
                const uint32_t nT = __ldg(&I->pois_n);
                const uint8_t* S = n.pois_start + (size_t)b * kPoissonBuckets;
                uint32_t words[8];
                philox_words8(n.seed, n.key0 + b, local0 >> 3, t, 1, words);
                const uint32_t wofs = local0 & 7u & ~(uint32_t)(NPT - 1);  // 0 for 8 per thread
#pragma unroll
                for (int k = 0; k < NPT; ++k) {
                    if (local0 + k >= nloc) continue;
                    float v = V[k];
                    uint32_t rk = r[k];
                    if (rk > 0) {
                        rk -= 1;
                        v = v_reset;
                    } else {
                        const uint32_t next = SPOIS ? poisson_count_s(Ts, Ss, nT, words[(wofs + k) & 7u])
                                                    : poisson_count(T, S, nT, words[(wofs + k) & 7u]);
                        const int32_t in = a0[k] + (int32_t)next * jext;
                        v = __fadd_rn(__fmul_rn(v, Pm), __fmul_rn(__int2float_rn(in), kLattice));
                        if (v >= v_th) {
                            spk |= 1u << k;
                            v = v_reset;
                            rk = R;
                        }
                    }
                    V[k] = v;
                    r[k] = (uint8_t)rk;
                }
                if (SYN == 1) {
                    // traces of the excitatory neurons: x decays and counts
                    // the arrivals of S_{t-d}; y decays and counts S_t
                    const uint32_t n_exc = __ldg(&I->n_exc);
                    const float Pp = __ldg(&I->Pp), Pn = __ldg(&I->Pn);
                    uint32_t arr = 0;
                    if (t >= n.d) {
                        const uint32_t slot = (uint32_t)((t - n.d) % n.D);
                        arr = (n.bits[(size_t)slot * (n.Np >> 5) + (id0 >> 5)] >> (id0 & 31u)) & ((1u << NPT) - 1u);
                    }
                    float xs[NPT], ys[NPT];
#pragma unroll
                    for (int h = 0; h < NPT / 4; ++h) {
                        *reinterpret_cast<float4*>(xs + 4 * h) = *reinterpret_cast<const float4*>(n.x + id0 + 4 * h);
                        *reinterpret_cast<float4*>(ys + 4 * h) = *reinterpret_cast<const float4*>(n.y + id0 + 4 * h);
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        if (local0 + k >= n_exc) continue;
                        float xv = __fmul_rn(xs[k], Pp);
                        if (arr >> k & 1u) xv = __fadd_rn(xv, 1.0f);
                        float yv = __fmul_rn(ys[k], Pn);
                        if (spk >> k & 1u) yv = __fadd_rn(yv, 1.0f);
                        xs[k] = xv;
                        ys[k] = yv;
                    }
#pragma unroll
                    for (int h = 0; h < NPT / 4; ++h) {
                        *reinterpret_cast<float4*>(n.x + id0 + 4 * h) = *reinterpret_cast<float4*>(xs + 4 * h);
                        *reinterpret_cast<float4*>(n.y + id0 + 4 * h) = *reinterpret_cast<float4*>(ys + 4 * h);
                    }
                }
                if (SYN == 2) {
                    // lazy: y is kept every step (its decayed value y(t-1) P-
                    // also goes to the ring slot of step t, where a pending
                    // depression finds it), the spike history shifts, and a
                    // row whose age reaches F is queued unless it transmits
                    // at this step (j in S_{t-d+1}), which replays it anyway
                    const uint32_t n_exc = __ldg(&I->n_exc);
                    const float Pn = __ldg(&I->Pn);
                    uint32_t tx = spk;
                    if (n.d > 1) {
                        tx = 0;
                        if (t + 1 >= n.d) {
                            const uint32_t slot = (uint32_t)((t + 1 - n.d) % n.D);
                            tx = (n.bits[(size_t)slot * (n.Np >> 5) + (id0 >> 5)] >> (id0 & 31u)) & ((1u << NPT) - 1u);
                        }
                    }
                    float ys[NPT], yp[NPT];
                    ulonglong2 hs[NPT];  // 128-bit histories: .x bits 0..63, .y bits 64..127
                    uint32_t ag[NPT];
#pragma unroll
                    for (int h = 0; h < NPT / 4; ++h) {
                        *reinterpret_cast<float4*>(ys + 4 * h) = *reinterpret_cast<const float4*>(n.y + id0 + 4 * h);
                        *reinterpret_cast<uint4*>(ag + 4 * h) = *reinterpret_cast<const uint4*>(n.age + id0 + 4 * h);
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) hs[k] = *reinterpret_cast<const ulonglong2*>(n.hist + 2 * (id0 + k));
                    const uint32_t t31 = (uint32_t)t & 0x7fffffffu;
#pragma unroll
                    for (int k = 0; k < NPT; ++k) {
                        yp[k] = 0.0f;
                        if (local0 + k >= n_exc) continue;
                        const float yd = __fmul_rn(ys[k], Pn);
                        yp[k] = yd;
                        ys[k] = (spk >> k & 1u) ? __fadd_rn(yd, 1.0f) : yd;
                        hs[k].y = (hs[k].y << 1) | (hs[k].x >> 63);
                        hs[k].x = (hs[k].x << 1) | (unsigned long long)(spk >> k & 1u);
                        const uint32_t lag = (t31 - (ag[k] & 0x7fffffffu)) & 0x7fffffffu;  // t - age
                        if (lag + 1u >= n.F && !(tx >> k & 1u)) xexp |= 1u << k;
                    }
                    float* yr = n.yring + (size_t)(t % n.F) * n.Np;
#pragma unroll
                    for (int h = 0; h < NPT / 4; ++h) {
                        *reinterpret_cast<float4*>(n.y + id0 + 4 * h) = *reinterpret_cast<float4*>(ys + 4 * h);
                        *reinterpret_cast<float4*>(yr + id0 + 4 * h) = *reinterpret_cast<float4*>(yp + 4 * h);
                    }
#pragma unroll
                    for (int k = 0; k < NPT; ++k) *reinterpret_cast<ulonglong2*>(n.hist + 2 * (id0 + k)) = hs[k];
                }
            }
            have = true;
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

    const uint32_t lane = lane_id();
    const uint32_t slot_q = (uint32_t)(t % n.D);
    const uint32_t slot_c = (uint32_t)(t & (n.cr - 1));
    if (SYN != 0) {
        // 32 / NPT lanes cover one 32-neuron bitmask word
        constexpr uint32_t L = 32 / NPT;
        uint32_t word = spk << (NPT * (lane & (L - 1u)));
#pragma unroll
        for (uint32_t o = 1; o < L; o <<= 1) word |= __shfl_xor_sync(kFull, word, o);
        if (active && (lane & (L - 1u)) == 0) n.bits[(size_t)slot_q * (n.Np >> 5) + (id0 >> 5)] = word;
    }
    if (SYN == 2) {
        // expiring rows -> xq: warp scan, one atomicAdd per warp that has any
        const uint32_t cx = __popc(xexp);
        uint32_t ix = cx;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, ix, o);
            if (lane >= (uint32_t)o) ix += v;
        }
        const uint32_t tot = __shfl_sync(kFull, ix, 31);
        if (tot) {
            uint32_t xb = 0;
            if (lane == 31) xb = atomicAdd(&n.xcount[t & 1ull], tot);
            xb = __shfl_sync(kFull, xb, 31) + ix - cx;
            uint32_t m = xexp;
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                n.xq[xb++] = id0 + bit;
            }
        }
    }
    // warp compaction: exclusive scan of the per-thread spike counts, one
    // atomicAdd on the instance's queue index
    const uint32_t c = __popc(spk);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(kFull, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    uint32_t wbase = 0;
    if (lane == 31 && total) wbase = atomicAdd(&n.icount[(size_t)slot_c * n.n_inst + b], total);
    // the state goes back while the atomic is in flight
    if (have) {
#pragma unroll
        for (int h = 0; h < NPT / 4; ++h) {
            *reinterpret_cast<float4*>(n.V + id0 + 4 * h) = *reinterpret_cast<float4*>(V + 4 * h);
            *reinterpret_cast<uint32_t*>(n.r + id0 + 4 * h) = *reinterpret_cast<uint32_t*>(r + 4 * h);
            *reinterpret_cast<int4*>(acc0 + id0 + 4 * h) = make_int4(0, 0, 0, 0);
        }
    }
    if (total == 0) return;
    const LogSlot L = spk ? log_slot(n, t, b) : LogSlot{0ull, 0ull, 0ull};
    wbase = __shfl_sync(kFull, wbase, 31);
    if (spk) file_spikes(n, t, id0, spk, incl - c, slot_q, pbase, wbase, L);
}

template <int MODEL, int SYN, bool STATS, int NPT>
__global__ void __launch_bounds__(256, (MODEL == 1 && SYN == 0) ? 5 : 1) k_update(Net n)
{
    const unsigned long long t = n.ctl->t + n.k;
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    step_bookkeeping(n, t, g, SYN == 2);
    // a receive launched as this kernel's programmatic dependent may start
    // (it waits for this kernel before touching what it writes)
    if (threadIdx.x == 0) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    update_neurons<MODEL, SYN, STATS, NPT, true>(n, t, g, n.acc0);
}

// Raster readout: chunks of instances' log regions (a chunk: len entries
// from log index src, instance inst, written at key index dst) -> sortable
// keys (step - t0) << 32 | global id, one block per chunk.
struct LogChunk {
    unsigned long long src, dst;
    uint32_t len, inst;
};

__global__ void k_raster_keys(Net n, const LogChunk* __restrict__ chunks, uint64_t t0, unsigned long long* __restrict__ keys)
{
    const LogChunk C = chunks[blockIdx.x];
    const uint32_t pbase = n.inst[C.inst].pbase, goff = n.inst[C.inst].goff;
    for (uint32_t i = threadIdx.x; i < C.len; i += blockDim.x) {
        const unsigned long long v = n.log[C.src + i];
        keys[C.dst + i] = (((v >> 32) - t0) << 32) | (unsigned long long)((uint32_t)v - pbase + goff);
    }
}

// Per instance b, the first entries of its log region (avail[b] entries in
// step order) at steps >= t0 and >= t1, by bisection: out[2b], out[2b+1].
__global__ void k_log_ranges(Net n, const unsigned long long* __restrict__ avail, uint64_t t0, uint64_t t1,
                             unsigned long long* __restrict__ out)
{
    for (uint32_t b = blockIdx.x * blockDim.x + threadIdx.x; b < n.n_inst; b += gridDim.x * blockDim.x) {
        const unsigned long long lo0 = n.inst[b].log_lo, m = avail[b];
        for (int e = 0; e < 2; ++e) {
            const uint64_t t = e ? t1 : t0;
            unsigned long long lo = 0, hi = m;
            while (lo < hi) {
                const unsigned long long mid = (lo + hi) / 2;
                if ((n.log[lo0 + mid] >> 32) < t)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            out[2 * b + e] = lo;
        }
    }
}

// Sorted keys -> steps and global ids.
__global__ void k_raster_split(const unsigned long long* __restrict__ keys, uint64_t count, uint64_t t0,
                               uint32_t* __restrict__ steps, uint32_t* __restrict__ ids)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (uint64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = keys[i];
        steps[i] = (uint32_t)((k >> 32) + t0);
        ids[i] = (uint32_t)k;
    }
}

// The step counter advances once per captured graph (the kernels of a graph
// carry their offset inside it); the per-step bookkeeping is done by the
// next step's update kernel.
__global__ void k_advance(Ctl* ctl, uint32_t steps) { ctl->t += steps; }

// Visit the spikes of one queue slot cut into K = 2^lk pieces each, K the
// largest power of two up to 16 that still leaves every warp of the grid
// one piece: f(j, c, lk) for piece c of spike j, a warp per piece.  With a
// few hundred spikes per step a warp per whole row would walk it alone.
template <class F>
__device__ __forceinline__ void for_each_piece(const Net& n, unsigned long long ts, F f)
{
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    const uint32_t* qs = n.q + (size_t)(ts % n.D) * n.Np;
    const unsigned int* ic = n.icount + (size_t)(ts & (n.cr - 1)) * n.n_inst;
    uint32_t total = 0;
    for (uint32_t b = 0; b < n.n_inst; ++b) total += ic[b];
    uint32_t lk = 0;
    while (lk < 4 && ((uint64_t)total << (lk + 1)) <= nwarps) ++lk;
    uint64_t u = warp;  // unit: piece u & (K - 1) of spike u >> lk, instance by instance
    uint32_t base = 0;
    for (uint32_t b = 0; b < n.n_inst; ++b) {
        const uint32_t cnt = ic[b];
        if ((u >> lk) < base + cnt) {
            const uint32_t* qb = qs + __ldg(&n.inst[b].pbase);
            for (; (u >> lk) < base + cnt; u += nwarps) f(qb[(u >> lk) - base], (uint32_t)(u & ((1u << lk) - 1u)), lk);
        }
        base += cnt;
    }
}

// Piece c of 2^lk of the index range [beg, end).
__device__ __forceinline__ void piece_of(uint64_t beg, uint64_t end, uint32_t c, uint32_t lk, uint64_t& pb, uint64_t& pe)
{
    const uint64_t len = end - beg;
    pb = beg + ((len * c) >> lk);
    pe = beg + ((len * (c + 1)) >> lk);
}

// ---------------------------------------------------------------------------
// Receive Spikes (Section III-A-2), global-accumulator form: a warp per
// piece of the rows of S_{t-d+1} (for_each_piece) walks it with coalesced
// target/weight loads and adds the weights with red.global.add into the
// L2-resident int32 accumulators of the targets (order-independent integer
// sums).
// ---------------------------------------------------------------------------
// ROWW: every row carries one weight (the source population's, as in the
// paper's models: Section III-A-2, Table 2), held per row in n.roww, so the
// walk reads the 4-byte targets alone.
template <bool W16, bool ROWW>
__device__ __forceinline__ void receive_global(const Net& n, unsigned long long t)
{
    if (t + 1 < n.d) return;
    const uint32_t lane = lane_id();
    unsigned long long ev = 0;
    for_each_piece(n, t + 1 - n.d, [&](uint32_t j, uint32_t c, uint32_t lk) {
        uint64_t pb, pe;
        piece_of(__ldg(n.roff + j), __ldg(n.roff + j + 1), c, lk, pb, pe);
        const uint32_t meta = __ldg(n.meta + j);
        const uint32_t shift = meta & 31u;
        const int32_t rw = ROWW ? __ldg(n.roww + j) : 0;
        int32_t* acc = (meta & 0x80u) ? n.acc1 : n.acc0;
        ev += pe - pb;
        uint64_t e = pb + lane;
        for (; e + 96 < pe; e += 128) {
            uint32_t tg[4];
            int32_t wv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                tg[k] = __ldg(n.tgt + e + 32 * k);
                wv[k] = ROWW ? rw
                             : (W16 ? ((int32_t)__ldg(n.w16 + e + 32 * k) << shift)
                                    : __float2int_rz(__ldg(n.w32 + e + 32 * k)));
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(acc + tg[k], wv[k]);
        }
        for (; e < pe; e += 32) {
            const uint32_t tg = __ldg(n.tgt + e);
            const int32_t wv = ROWW ? rw : (W16 ? ((int32_t)__ldg(n.w16 + e) << shift) : __float2int_rz(__ldg(n.w32 + e)));
            atomicAdd(acc + tg, wv);
        }
    });
    if (lane == 0 && ev) atomicAdd(&n.ctl->events, ev);
}

template <bool W16, bool ROWW>
__global__ void __launch_bounds__(256) k_receive_global(Net n)
{
    receive_global<W16, ROWW>(n, n.ctl->t + n.k);
}

// ---------------------------------------------------------------------------
// Update Synapses (Section III-A-1), pair STDP on exc -> exc synapses.
// Depression for the rows of S_{t-d} (the presynaptic spikes reaching their
// synapses at step t), run before the neuron update of step t so that the
// postsynaptic trace it reads is y(t-1), decayed here by one step.
// ---------------------------------------------------------------------------
template <bool W16>
__global__ void __launch_bounds__(256) k_stdp_depress(Net n)
{
    const unsigned long long t = n.ctl->t + n.k;
    if (t < n.d) return;
    const uint32_t lane = lane_id();
    for_each_piece(n, t - n.d, [&](uint32_t j, uint32_t c, uint32_t lk) {
        const uint32_t meta = __ldg(n.meta + j);
        if (!(meta & 0x40u)) return;  // inhibitory source: no plastic synapses
        const InstDev* I = n.inst + __ldg(n.inst_of_w32 + (j >> 5));
        const uint32_t pbase = __ldg(&I->pbase), n_exc = __ldg(&I->n_exc);
        const float Pn = __ldg(&I->Pn), Am = __ldg(&I->Am);
        const int32_t wmax = __ldg(&I->wmax);
        uint64_t beg, end;
        piece_of(__ldg(n.roff + j), __ldg(n.roff + j + 1), c, lk, beg, end);
        for (uint64_t e = beg + lane; e < end; e += 32) {
            const uint32_t i = __ldg(n.tgt + e);
            if (i - pbase >= n_exc) continue;
            const float yd = __fmul_rn(n.y[i], Pn);
            const int32_t dw = __float2int_rn(__fmul_rn(Am, yd));
            if (W16) {
                const int32_t w = min(max((int32_t)n.w16[e] + dw, 0), wmax);
                n.w16[e] = (int16_t)w;
            } else {
                const int32_t w = min(max(__float2int_rz(n.w32[e]) + dw, 0), wmax);
                n.w32[e] = (float)w;
            }
        }
    });
}

// Potentiation for the in-edges of the excitatory spikers of S_t, after the
// neuron update of step t (the presynaptic traces then include step t's
// arrivals, so a coincident arrival counts as causal).
template <bool W16>
__global__ void __launch_bounds__(256) k_stdp_potentiate(Net n)
{
    const unsigned long long t = n.ctl->t + n.k;
    const uint32_t lane = lane_id();
    for_each_piece(n, t, [&](uint32_t i, uint32_t c, uint32_t lk) {
        const InstDev* I = n.inst + __ldg(n.inst_of_w32 + (i >> 5));
        const float Ap = __ldg(&I->Ap);
        const int32_t wmax = __ldg(&I->wmax);
        uint64_t beg, end;
        piece_of(__ldg(n.coff + i), __ldg(n.coff + i + 1), c, lk, beg, end);
        for (uint64_t k = beg + lane; k < end; k += 32) {
            const uint32_t e = __ldg(n.cedge + k);
            const uint32_t j = __ldg(n.cpre + k);
            const int32_t dw = __float2int_rn(__fmul_rn(Ap, n.x[j]));
            if (W16) {
                const int32_t w = min(max((int32_t)n.w16[e] + dw, 0), wmax);
                n.w16[e] = (int16_t)w;
            } else {
                const int32_t w = min(max(__float2int_rz(n.w32[e]) + dw, 0), wmax);
                n.w32[e] = (float)w;
            }
        }
    });
}

// ---------------------------------------------------------------------------
// Lazy Update Synapses (Section III-A-1).  The exc -> exc synapses of a row
// stay stale until the row transmits a spike (it is in S_{t-d+1}) or until
// its age reaches the history length F; then one block brings the whole row
// up to date in registers.  All synapses of a row share their age (they
// transmit together), so one age per row is kept: a = the first step whose
// events the row has not seen, with the presynaptic trace stored as x(a-1).
// The pass replays, per synapse j -> i, the eager rule's events of steps
// a..t in their order: the depression of step a if j's spike arrived then
// (an arrival follows a transmission by one step, and a transmission always
// brings the row up to date, so only step a can hold one: a flag records
// it), with y_i(a-1) P- from the ring, then the potentiation of every step
// s in a..t at which i spiked (bit t - s of i's 128-bit history), with x_j(s).
// The row's x(s) sequence is the eager one, one rounded multiply per step.
// ---------------------------------------------------------------------------
constexpr int kLazyMaxF = 128;   // longest history (steps): the bits of the two history words
constexpr int kLazyThreads = 256;
constexpr int kLazyBatch = 4;    // edges per thread with their loads in flight together

// The row-level part of a replay: the window of steps and the constants
// every synapse of the row uses.
struct LazyRow {
    uint32_t pbase, n_exc, L;
    float Ap, Am;
    int32_t wmax;
    bool arrived;
    unsigned long long win_lo, win_hi;  // history bits of steps a..t (bits 0 .. L-1 of the 128)
    const float* yr;          // ring slot of step a (when arrived)
};

__device__ __forceinline__ LazyRow lazy_row(const Net& n, uint32_t j, uint32_t ag, unsigned long long t, bool leader)
{
    LazyRow r;
    const InstDev* I = n.inst + __ldg(n.inst_of_w32 + (j >> 5));
    r.pbase = __ldg(&I->pbase);
    r.n_exc = __ldg(&I->n_exc);
    r.Ap = __ldg(&I->Ap);
    r.Am = __ldg(&I->Am);
    r.wmax = __ldg(&I->wmax);
    r.arrived = (ag >> 31) != 0;
    uint32_t L = ((((uint32_t)t & 0x7fffffffu) - (ag & 0x7fffffffu)) & 0x7fffffffu) + 1u;  // steps a..t
    if (L > n.F) {  // the history no longer covers the row: report, and stay inside the buffers
        if (leader) atomicOr(&n.ctl->err, kErrLazyAge);
        L = n.F;
    }
    r.L = L;
    r.win_lo = L >= 64u ? ~0ull : (1ull << L) - 1ull;
    r.win_hi = L <= 64u ? 0ull : (L >= 128u ? ~0ull : (1ull << (L - 64u)) - 1ull);
    // the ring slot of step a = t - (L - 1): an arrival implies a >= 1
    r.yr = r.arrived ? n.yring + (size_t)((t - (L - 1u)) % n.F) * n.Np : nullptr;
    return r;
}

// x(s) for s = a..t into xs[0..L), one rounded multiply per step (the
// arrival of step a, if any, added after its decay); one thread.
__device__ __forceinline__ void lazy_trajectory(const Net& n, uint32_t j, const LazyRow& r, float* xs)
{
    const float Pp = __ldg(&n.inst[__ldg(n.inst_of_w32 + (j >> 5))].Pp);
    float x = n.x[j];
    for (uint32_t k = 0; k < r.L; ++k) {
        x = __fmul_rn(x, Pp);
        if (k == 0 && r.arrived) x = __fadd_rn(x, 1.0f);
        xs[k] = x;
    }
}

// Targets of B synapses, `stride` apart from e0 (past the end: an id that is
// never plastic, since pbase + n_exc < 2^31).
template <int B>
__device__ __forceinline__ void lazy_targets(const Net& n, uint64_t e0, uint64_t end, uint32_t stride, uint32_t* ii)
{
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const uint64_t e = e0 + (uint64_t)u * stride;
        ii[u] = e < end ? __ldg(n.tgt + e) : 0xffffffffu;
    }
}

// Replay B synapses whose targets are loaded: the weights, the pending
// arrival's traces and the targets' histories are loaded at once,
// then (after `sync`: the block waits for the trajectory) each synapse takes
// the depression of the pending arrival and the potentiation of every step
// at which its target spiked, in step order, each change clipped to
// [0, w_max]; changed weights only are written back.
template <bool W16, int B>
__device__ __forceinline__ void lazy_apply(const Net& n, const LazyRow& r, const float* xs, const uint32_t* ii,
                                           uint64_t e0, uint32_t stride, bool sync)
{
    int32_t w0[B];
    float yv[B];
    ulonglong2 hm[B];
#pragma unroll
    for (int u = 0; u < B; ++u) {
        w0[u] = 0;
        yv[u] = 0.0f;
        hm[u] = make_ulonglong2(0ull, 0ull);
        if (ii[u] - r.pbase < r.n_exc) {  // excitatory target: plastic
            const uint64_t e = e0 + (uint64_t)u * stride;
            w0[u] = W16 ? (int32_t)n.w16[e] : __float2int_rz(n.w32[e]);
            if (r.arrived) yv[u] = r.yr[ii[u]];
            hm[u] = *reinterpret_cast<const ulonglong2*>(n.hist + 2 * (size_t)ii[u]);
            hm[u].x &= r.win_lo;
            hm[u].y &= r.win_hi;
        }
    }
    if (sync) __syncthreads();
#pragma unroll
    for (int u = 0; u < B; ++u) {
        if (ii[u] - r.pbase >= r.n_exc) continue;
        int32_t w = w0[u];
        if (r.arrived) w = min(max(w + __float2int_rn(__fmul_rn(r.Am, yv[u])), 0), r.wmax);
        // the older word first; in each, the earliest remaining step (t - k) first
        unsigned long long m = hm[u].y;
        while (m) {
            const int k = 63 - __clzll((long long)m);
            m ^= 1ull << k;
            w = min(max(w + __float2int_rn(__fmul_rn(r.Ap, xs[r.L - 65u - (uint32_t)k])), 0), r.wmax);
        }
        m = hm[u].x;
        while (m) {
            const int k = 63 - __clzll((long long)m);
            m ^= 1ull << k;
            w = min(max(w + __float2int_rn(__fmul_rn(r.Ap, xs[r.L - 1u - (uint32_t)k])), 0), r.wmax);
        }
        if (w != w0[u]) {
            const uint64_t e = e0 + (uint64_t)u * stride;
            if (W16)
                n.w16[e] = (int16_t)w;
            else
                n.w32[e] = (float)w;
        }
    }
}

__device__ __forceinline__ uint32_t lazy_new_age(unsigned long long t, bool transmit)
{
    return (uint32_t)((t + 1) & 0x7fffffffull) | (transmit ? 0x80000000u : 0u);
}

// One row by the whole block (every thread calls it with the same row): the
// first batch of targets is in flight while thread 0 computes the
// trajectory; the block waits for it once; the row's age and x change after
// every thread has read them.
template <bool W16>
__device__ __forceinline__ void lazy_replay_row(const Net& n, uint32_t j, uint32_t ag, uint64_t beg, uint64_t end,
                                                unsigned long long t, bool transmit, float* xs)
{
    constexpr int B = kLazyBatch;
    const uint32_t tid = threadIdx.x;
    const LazyRow r = lazy_row(n, j, ag, t, tid == 0);
    uint64_t e0 = beg + tid;
    uint32_t ii[B];
    lazy_targets<B>(n, e0, end, kLazyThreads, ii);
    if (tid == 0) lazy_trajectory(n, j, r, xs);
    lazy_apply<W16, B>(n, r, xs, ii, e0, kLazyThreads, true);
    for (e0 += (uint64_t)B * kLazyThreads; e0 < end; e0 += (uint64_t)B * kLazyThreads) {  // longer rows
        lazy_targets<B>(n, e0, end, kLazyThreads, ii);
        lazy_apply<W16, B>(n, r, xs, ii, e0, kLazyThreads, false);
    }
    __syncthreads();
    if (tid == 0) {
        n.age[j] = lazy_new_age(t, transmit);
        n.x[j] = xs[r.L - 1u];
    }
}

// The rows one lazy step replays, in a fixed order: the spikers of
// S_{t-d+1} instance by instance (inhibitory ones included; they are
// skipped), then the expiry queue.  at(r) returns row r; r must not
// decrease between calls.
struct LazyRows {
    const Net* n;
    const uint32_t* qs;       // queue slot of S_{t-d+1} (null before step d-1)
    const unsigned int* ic;   // its per-instance counts
    uint32_t b, base;         // current instance and the rows before it
    uint32_t n_tx, n_x;       // rows of the two sets

    __device__ __forceinline__ void init(const Net& net, unsigned long long t)
    {
        n = &net;
        qs = nullptr;
        ic = nullptr;
        b = 0;
        base = 0;
        n_tx = 0;
        if (t + 1 >= net.d) {
            const unsigned long long ts = t + 1 - net.d;
            qs = net.q + (size_t)(ts % net.D) * net.Np;
            ic = net.icount + (size_t)(ts & (net.cr - 1)) * net.n_inst;
            for (uint32_t k = 0; k < net.n_inst; ++k) n_tx += ic[k];
        }
        n_x = min(net.xcount[t & 1ull], net.Np);
    }
    __device__ __forceinline__ uint32_t total() const { return n_tx + n_x; }
    __device__ __forceinline__ uint32_t at(uint32_t r)
    {
        if (r >= n_tx) return n->xq[r - n_tx];
        while (r >= base + ic[b]) base += ic[b++];
        return qs[__ldg(&n->inst[b].pbase) + (r - base)];
    }
};

// One step of lazy Update Synapses, after the neuron update of step t and
// before the receive: the excitatory rows of S_{t-d+1} (they transmit now,
// with Syn_{t+1}) and the rows of the expiry queue, a block per row.  The
// two sets are disjoint (the update queues no transmitting row), so every
// row is replayed once.  The next row's record is loaded while the current
// one is replayed.
template <bool W16>
__global__ void __launch_bounds__(kLazyThreads, 4) k_stdp_lazy(Net n)
{
    __shared__ float xs[kLazyMaxF];
    const unsigned long long t = n.ctl->t + n.k;
    LazyRows rows;
    rows.init(n, t);
    const uint32_t R = rows.total();
    uint32_t r = blockIdx.x;
    if (r >= R) return;
    uint32_t j = rows.at(r);
    uint32_t meta = __ldg(n.meta + j), ag = n.age[j];
    uint64_t beg = __ldg(n.roff + j), end = __ldg(n.roff + j + 1);
    for (;;) {
        const bool transmit = r < rows.n_tx;
        const uint32_t rn = r + gridDim.x;  // the next row's record
        uint32_t jn = 0, metan = 0, agn = 0;
        uint64_t begn = 0, endn = 0;
        if (rn < R) {
            jn = rows.at(rn);
            metan = __ldg(n.meta + jn);
            agn = n.age[jn];
            begn = __ldg(n.roff + jn);
            endn = __ldg(n.roff + jn + 1);
        }
        if (meta & 0x40u) lazy_replay_row<W16>(n, j, ag, beg, end, t, transmit, xs);  // excitatory source
        if (rn >= R) break;
        r = rn;
        j = jn;
        meta = metan;
        ag = agn;
        beg = begn;
        end = endn;
    }
}

// Bring every stale excitatory row up to date after step `now` (between
// steps, before the weights or x are read or written), a block per row.  A
// row that transmitted at `now` is already current (its age is now + 1).
template <bool W16>
__global__ void __launch_bounds__(kLazyThreads) k_stdp_flush(Net n, unsigned long long now)
{
    __shared__ float xs[kLazyMaxF];
    const uint32_t cur = (uint32_t)((now + 1) & 0x7fffffffull);
    for (uint32_t j = blockIdx.x; j < n.Np; j += gridDim.x) {
        if (!(__ldg(n.meta + j) & 0x40u)) continue;
        const uint32_t ag = n.age[j];
        if ((ag & 0x7fffffffu) == cur) continue;
        lazy_replay_row<W16>(n, j, ag, __ldg(n.roff + j), __ldg(n.roff + j + 1), now, false, xs);
    }
}

// ---------------------------------------------------------------------------
// Init stage (Fig. 1 caption): N -> N_0.
// ---------------------------------------------------------------------------
// With lazy plasticity a row's age starts at -(local id mod F) (mod 2^31):
// the steps before 0 hold no events, and the staggered ages spread the rows'
// expiries over F steps instead of replaying every row at once.
__global__ void k_init_state(Net n, int vogels, int stdp, int lazy)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= (n.Np >> 3)) return;
    const uint32_t id0 = g * 8u;
    const uint32_t b = n.inst_of_w32[g >> 2];
    const InstDev* I = n.inst + b;
    const uint32_t local0 = id0 - I->pbase;
    uint32_t words[8];
    philox_words8(n.seed, n.key0 + b, local0 >> 3, 0, 0, words);
    for (int k = 0; k < 8; ++k) {
        const uint32_t id = id0 + k;
        float v = 0.0f;
        if (local0 + k < I->n) {
            const float u01 = __fmul_rn(__uint2float_rn(words[k] >> 8), 1.0f / 16777216.0f);
            v = __fadd_rn(I->v0_lo, __fmul_rn(I->v0_span, u01));
        }
        n.V[id] = v;
        n.r[id] = 0;
        n.acc0[id] = 0;
        if (vogels) {
            n.ge[id] = 0.0f;
            n.gi[id] = 0.0f;
            n.acc1[id] = 0;
        }
        if (stdp) {
            n.x[id] = 0.0f;
            n.y[id] = 0.0f;
        }
        if (lazy) n.age[id] = (0u - (local0 + k) % n.F) & 0x7fffffffu;
    }
}

// ---------------------------------------------------------------------------
// Graph set-up: one warp per row.  Maps targets to padded ids (checking that
// they stay inside the source's instance), picks the row's weight shift and
// writes the stored weights.
// ---------------------------------------------------------------------------
// STDP column index (eager potentiation): the plastic (exc -> exc) in-edges
// of every padded post id, as a counting sort on the device.  k_col_count
// counts them per post id (cnt[Np], zeroed), an exclusive scan of cnt gives
// the column offsets, k_col_fill files each edge (its index, its padded
// source) at its post id's next slot (cur: a copy of the offsets).  The
// order inside a column is the order the atomics hand out; potentiation
// updates every edge of a column on its own, so results do not depend on it.
// A warp per row; tgt holds padded ids, meta bit 6 marks an excitatory source.
__global__ void k_col_count(Net n, unsigned long long* __restrict__ cnt)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < n.Np; pj += nwarps) {
        if (!(n.meta[pj] & 0x40u)) continue;
        const InstDev& I = n.inst[n.inst_of_w32[pj >> 5]];
        const uint32_t pb = I.pbase, ne = I.n_exc;
        for (uint64_t e = n.roff[pj] + lane; e < n.roff[pj + 1]; e += 32) {
            const uint32_t i = n.tgt[e];
            if (i - pb < ne) atomicAdd(cnt + i, 1ull);
        }
    }
}

__global__ void k_col_fill(Net n, unsigned long long* __restrict__ cur, uint32_t* __restrict__ cedge,
                           uint32_t* __restrict__ cpre)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < n.Np; pj += nwarps) {
        if (!(n.meta[pj] & 0x40u)) continue;
        const InstDev& I = n.inst[n.inst_of_w32[pj >> 5]];
        const uint32_t pb = I.pbase, ne = I.n_exc;
        for (uint64_t e = n.roff[pj] + lane; e < n.roff[pj + 1]; e += 32) {
            const uint32_t i = n.tgt[e];
            if (i - pb < ne) {
                const unsigned long long k = atomicAdd(cur + i, 1ull);
                cedge[k] = (uint32_t)e;
                cpre[k] = pj;
            }
        }
    }
}

// One weight per row spread over the row's edges: w[e] = w_row[row_src[pj]]
// for the edges e of padded row pj (row_src: the global id of a padded
// row, ~0 for padding, whose rows are empty).  A warp per row.
__global__ void k_spread_row_weights(const uint64_t* __restrict__ roff, const uint32_t* __restrict__ row_src,
                                     const int32_t* __restrict__ w_row, uint32_t Np, int32_t* __restrict__ w)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint64_t beg = roff[pj], end = roff[pj + 1];
        if (beg == end) continue;
        const int32_t x = w_row[row_src[pj]];
        for (uint64_t e = beg + lane; e < end; e += 32) w[e] = x;
    }
}

// The weight of every row whose edges all carry the same 16-bit code:
// roww[pj] = code << shift (0 for an empty row); *mixed is set when some row
// carries two or more codes.  A warp per row.
__global__ void k_row_weights(const uint64_t* __restrict__ roff, const int16_t* __restrict__ w16,
                              const uint8_t* __restrict__ meta, uint32_t Np, int32_t* __restrict__ roww,
                              unsigned int* mixed)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint64_t beg = roff[pj], end = roff[pj + 1];
        const int16_t w0 = beg < end ? w16[beg] : (int16_t)0;
        bool same = true;
        for (uint64_t e = beg + lane; e < end; e += 32) same = same && w16[e] == w0;
        if (!__all_sync(kFull, same) && lane == 0) atomicOr(mixed, 1u);
        if (lane == 0) roww[pj] = (int32_t)w0 << (meta[pj] & 31u);
    }
}

struct RowMapArgs {
    const uint64_t* roff;        // padded row offsets (Np+1)
    const uint32_t* row_src;     // padded id -> global id (or ~0u for padding)
    const uint32_t* row_inst;    // padded id -> instance
    const uint32_t* g_inst_off;  // global instance offsets (n_inst+1)
    const uint32_t* pbase;       // padded bases (n_inst)
    const uint32_t* n_exc;       // per instance
    uint32_t* tgt;               // in: global ids, out: padded ids
    const int32_t* wq;           // lattice weights
    int16_t* w16;
    float* w32;
    uint8_t* meta;
    uint32_t Np;
    int w16_mode, vogels, stdp;
    unsigned int* err;
    unsigned int* unsorted;      // set to 1 if some row's targets are not ascending
};

// smallest s with -32768 * 2^s <= w <= 32767 * 2^s (99 if none up to 15)
__device__ __forceinline__ int shift_needed(int32_t w)
{
    int s = 0;
    while ((long long)w > 32767LL * (1LL << s) || (long long)w < -32768LL * (1LL << s)) {
        if (++s > 15) return 99;
    }
    return s;
}

__global__ void k_map_rows(RowMapArgs a)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < a.Np; pj += nwarps) {
        const uint64_t beg = a.roff[pj], end = a.roff[pj + 1];
        const uint32_t j = a.row_src[pj];
        if (j == 0xffffffffu) {
            if (lane == 0) a.meta[pj] = 0;
            continue;
        }
        const uint32_t b = a.row_inst[pj];
        const uint32_t g0 = a.g_inst_off[b], g1 = a.g_inst_off[b + 1];
        const uint32_t pb = a.pbase[b];
        const bool exc = (j - g0) < a.n_exc[b];
        int s = 0;
        bool bad_t = false, bad_w = false;
        for (uint64_t e = beg + lane; e < end; e += 32) {
            const uint32_t tg = a.tgt[e];
            if (tg < g0 || tg >= g1) bad_t = true;
            const int32_t w = a.wq[e];
            if (a.w16_mode) {
                s = max(s, shift_needed(w));
            } else if (w > (1 << 24) || w < -(1 << 24)) {
                bad_w = true;
            }
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) s = max(s, __shfl_xor_sync(kFull, s, o));
        if (s > 15) bad_w = true;
        const uint32_t mask = s >= 31 ? 0xffffffffu : ((1u << s) - 1u);
        for (uint64_t e = beg + lane; e < end; e += 32) {
            const uint32_t tg = a.tgt[e];
            if (tg >= g0 && tg < g1) a.tgt[e] = tg - g0 + pb;
            const int32_t w = a.wq[e];
            if (a.w16_mode) {
                if (s <= 15 && ((uint32_t)w & mask)) bad_w = true;
                a.w16[e] = (int16_t)(s <= 15 ? (w >> s) : 0);
            } else {
                a.w32[e] = (float)w;
            }
        }
        __syncwarp();
        bool unsorted = false;
        for (uint64_t e = beg + 1 + lane; e < end; e += 32)
            if (a.tgt[e] < a.tgt[e - 1]) unsorted = true;
        if (__any_sync(kFull, unsorted) && lane == 0) atomicOr(a.unsorted, 1u);
        const bool any_bad_t = __any_sync(kFull, bad_t);
        const bool any_bad_w = __any_sync(kFull, bad_w);
        if (lane == 0) {
            if (any_bad_t) atomicOr(a.err, kErrBadTarget);
            if (any_bad_w) atomicOr(a.err, kErrBadWeight);
            if (a.stdp && exc && s != 0) atomicOr(a.err, kErrPlasticShift);
            a.meta[pj] = (uint8_t)((a.w16_mode ? s : 0) | (exc ? 0x40 : 0) | ((a.vogels && !exc) ? 0x80 : 0));
        }
    }
}

// Re-expand stored weights to int32 lattice units (CSR order).
__global__ void k_weights_out(const uint64_t* roff, const uint8_t* meta, const int16_t* w16, const float* w32,
                              int w16_mode, uint32_t Np, int32_t* out)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint64_t beg = roff[pj], end = roff[pj + 1];
        const uint32_t s = meta[pj] & 31u;
        for (uint64_t e = beg + lane; e < end; e += 32)
            out[e] = w16_mode ? ((int32_t)w16[e] << s) : __float2int_rz(w32[e]);
    }
}

__global__ void k_weights_in(const uint64_t* roff, const uint8_t* meta, const int32_t* in, int w16_mode,
                             uint32_t Np, int16_t* w16, float* w32, unsigned int* err)
{
    const uint32_t lane = lane_id();
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint64_t beg = roff[pj], end = roff[pj + 1];
        const uint32_t s = meta[pj] & 31u;
        for (uint64_t e = beg + lane; e < end; e += 32) {
            const int32_t w = in[e];
            if (w16_mode) {
                const int32_t c = w >> s;
                if ((c << s) != w || c > 32767 || c < -32768) atomicOr(err, kErrBadWeight);
                w16[e] = (int16_t)c;
            } else {
                w32[e] = (float)w;
            }
        }
    }
}

// Row records for the receive: start, length and meta of every padded row.
__global__ void k_row_info(const uint64_t* roff, const uint8_t* meta, uint32_t Np, uint4* rinfo)
{
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < Np; j += gridDim.x * blockDim.x) {
        const uint64_t a = roff[j], b = roff[j + 1];
        rinfo[j] = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)(b - a), meta[j]);
    }
}

// ---------------------------------------------------------------------------
// Diagnostics (binary64 reductions): population rate and mean ISI CV of one
// instance.  out[0] = spikes, out[1] = sum of CVs, out[2] = neurons with >= 3
// spikes.
// ---------------------------------------------------------------------------
__global__ void k_stats(const uint32_t* cnt, const unsigned long long* sum, const unsigned long long* sq,
                        uint32_t lo, uint32_t hi, double* out)
{
    double s_spk = 0.0, s_cv = 0.0, s_n = 0.0;
    for (uint32_t i = lo + blockIdx.x * blockDim.x + threadIdx.x; i < hi; i += gridDim.x * blockDim.x) {
        const uint32_t c = cnt[i];
        s_spk += (double)c;
        if (c >= 3) {
            const double m = (double)sum[i] / (double)(c - 1);
            const double var = (double)sq[i] / (double)(c - 1) - m * m;
            s_cv += sqrt(var > 0.0 ? var : 0.0) / m;
            s_n += 1.0;
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        s_spk += __shfl_xor_sync(kFull, s_spk, o);
        s_cv += __shfl_xor_sync(kFull, s_cv, o);
        s_n += __shfl_xor_sync(kFull, s_n, o);
    }
    if ((threadIdx.x & 31u) == 0) {
        atomicAdd(out + 0, s_spk);
        atomicAdd(out + 1, s_cv);
        atomicAdd(out + 2, s_n);
    }
}

}  // namespace snn
