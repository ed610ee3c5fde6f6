// snn_fused.cuh -- one kernel per timestep: Update Neurons and Receive Spikes
// of the same step side by side.
//
// With a delay of d >= 2 steps the two stages of a timestep touch disjoint
// data (Section III-A-1, Fig. 1): Update Neurons at step t reads the input
// that the receive of step t-1 accumulated and writes the spike queue S_t,
// while Receive Spikes at step t delivers S_{t-d+1}, a queue finished d-1
// steps earlier, into the input of step t+1.  Holding the input in two
// buffers, one per step parity (the update of step t reads and clears buffer
// t & 1, the receive of step t adds into buffer (t+1) & 1), removes the last
// ordering between them, so one persistent launch can run both: its CTAs
// take work units from one counter,
//
//   * the per-step plan of step t+1's receive (the one-block plan of
//     snn_tiled.cuh, which reads the spike counts of S_{t+2-d}: final before
//     this launch when d >= 3),
//   * the receive items of step t (heaviest first), each as in
//     k_receive_tiled (shared-memory accumulators, bulk copy or bulk
//     add-reduce into the input buffer),
//   * chunks of 4,096 neurons of the update (8 per thread, the fixed Brunel
//     update of snn_kernels.cuh with its warp compaction and raster log),
//
// so the update's arithmetic fills the issue slots the latency-bound receive
// leaves idle, and the update chunks even out the end of the receive.  The
// next step's kernel starts when this one ends (the launch boundary is the
// step's only synchronisation).  Results are those of the separate kernels,
// bit for bit: integer sums do not depend on the order of the adds, and
// every neuron is updated by the same binary32 operations.
#pragma once
#include <cuda_runtime.h>

#include "snn_device.cuh"
#include "snn_kernels.cuh"
#include "snn_tiled.cuh"

namespace snn {

constexpr int kFusedThreads = 512;    // two CTAs per SM, as the tiled receive
constexpr uint32_t kFusedChunk = kFusedThreads * kUpdateNeurons;  // neurons of one update unit

enum : uint32_t { kUnitPlan = 0, kUnitRecv = 1, kUnitUpdate = 2, kUnitDone = 3 };

struct FusedDev {
    const TileDev* tiles;
    const uint32_t* split;
    StepPlan plan[2];          // the plan of step s is plan[s & 1]
    uint32_t n_tiles, max_len;
    uint32_t n_ctas, cap, items_cap;  // the plan's inputs (n_ctas: this kernel's grid)
    uint32_t n_chunks;         // update units: ceil(Np / kFusedChunk)
    uint32_t lead;             // receive items taken before update units start to alternate with them
    uint32_t plan_bytes;       // shared memory the plan uses (cleared after it)
};

// One update chunk, compiled as a function of its own: inlined, its
// registers add to the receive's and the kernel spills at the 64 that two
// CTAs of 512 threads per SM allow; as a call each side keeps its own.
template <bool STATS>
__device__ __noinline__ void update_chunk(const Net& n, unsigned long long t, uint32_t g, int32_t* acc)
{
    update_neurons<1, 0, STATS, kUpdateNeurons>(n, t, g, acc);
}

// Work unit w of the step: the plan of the next step first, then the first
// `lead` receive items, then receive items and update chunks alternately
// while both last, then what is left of either.
__device__ __forceinline__ void fused_unit(const FusedDev& F, uint32_t n_items, uint32_t w, uint32_t& kind,
                                           uint32_t& idx)
{
    if (w == 0) {
        kind = kUnitPlan;
        idx = 0;
        return;
    }
    w -= 1;
    const uint32_t L = min(F.lead, n_items);
    if (w < L) {
        kind = kUnitRecv;
        idx = w;
        return;
    }
    w -= L;
    const uint32_t rR = n_items - L, nU = F.n_chunks, m = min(rR, nU);
    if (w < 2 * m) {
        kind = (w & 1u) ? kUnitUpdate : kUnitRecv;
        idx = (w & 1u) ? (w >> 1) : L + (w >> 1);
        return;
    }
    w -= 2 * m;
    if (w < rR - m) {
        kind = kUnitRecv;
        idx = L + m + w;
    } else if (w < (rR - m) + (nU - m)) {
        kind = kUnitUpdate;
        idx = m + (w - (rR - m));
    } else {
        kind = kUnitDone;
        idx = 0;
    }
}

// One timestep of the Brunel model without plasticity (delay >= 3), packed or
// unpacked 16-bit edges (WM), optional spike statistics.
template <int WM, bool STATS>
__global__ void __launch_bounds__(kFusedThreads, 2) k_step_fused(Net n, FusedDev F)
{
    extern __shared__ __align__(16) int32_t acc_s[];  // max(max_len words, the plan's bytes)
    __shared__ TileDev s_T[2];
    __shared__ ItemDev s_I[2];
    __shared__ uint32_t s_kind[2], s_idx[2];
    const unsigned long long t = n.ctl->t + n.k;
    const uint32_t tid = threadIdx.x, lane = tid & 31u;
    const bool odd = (t & 1ull) != 0;
    // the input buffers of this step (taken where used, to keep registers
    // free): the update reads and clears buffer t & 1, the receive adds into
    // buffer (t+1) & 1, which the next step's update reads
    const unsigned long long pol = evict_first_policy();
    unsigned long long ev = 0;  // every lane of a warp counts the warp's segments; lane 0 reports
    bool bad = false;

    // the bookkeeping of the previous step, once (CTA 0)
    if (blockIdx.x == 0)
        for (uint32_t gt = tid; gt < max(n.n_inst, 1u); gt += blockDim.x) step_bookkeeping(n, t, gt, false);

    const uint32_t n_items = t + 1 >= n.d ? (odd ? F.plan[1].hdr : F.plan[0].hdr)[0] : 0u;
    // unit w's record into buffer b (thread 0)
    auto take = [&](uint32_t w, uint32_t b) {
        uint32_t kind, idx;
        fused_unit(F, n_items, w, kind, idx);
        if (kind == kUnitRecv) {
            const ItemDev I = (odd ? F.plan[1].items : F.plan[0].items)[idx];
            if (I.k < F.n_tiles && I.s_beg <= I.s_end) {
                s_I[b] = I;
                s_T[b] = F.tiles[I.k];
            } else {  // not produced by a correct plan: report, touch nothing
                atomicOr(&n.ctl->err, kErrPlan);
                kind = kUnitDone;
            }
        }
        s_kind[b] = kind;
        s_idx[b] = idx;
    };
    if (tid == 0) take(blockIdx.x, 0);
    // the accumulators start at zero, and every unit leaves them at zero
    {
        const uint32_t words = max(F.max_len, (F.plan_bytes + 3u) / 4u);
        for (uint32_t i = tid; i < (words + 3u) / 4u; i += blockDim.x)
            reinterpret_cast<int4*>(acc_s)[i] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    for (uint32_t b = 0; s_kind[b] != kUnitDone; b ^= 1u) {
        const uint32_t kind = s_kind[b];
        if (kind == kUnitRecv) {
            const ItemDev& I = s_I[b];
            const TileDev& T = s_T[b];
            const unsigned long long ts = t + 1 - n.d;  // a receive item exists only when t + 1 >= d
            deliver_pipe<WM, 1>(n, T, n.q + (size_t)(ts % n.D) * n.Np + T.pbase, T.pbase, F.split + T.split, acc_s,
                                I.s_beg, I.s_end, pol, ev, bad);
            if (tid == 0) take(atomicAdd(n.tile_ctr + (t & 1ull), 1u) + gridDim.x, b ^ 1u);
            // the tile's input for the next update, or this part's share of
            // it: the shared-memory adds are made visible to the copy engine,
            // which reads them out before they are cleared
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            {  // warp w copies out and clears slice w of the len words (multiples of 16)
                const uint32_t nwarps = blockDim.x >> 5, warp = tid >> 5;
                const uint32_t chunks = T.len / 16u, cpw = (chunks + nwarps - 1) / nwarps, c0 = warp * cpw;
                const uint32_t per = c0 < chunks ? 16u * min(cpw, chunks - c0) : 0u, w0 = 16u * c0;
                if (lane == 0 && per) {
                    bulk_out((odd ? n.acc0 : n.accx) + T.lo + w0, acc_s + w0, per * 4u, I.P > 1);
                    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                    asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
                }
                __syncwarp();
                for (uint32_t i = lane; i < per / 4; i += 32)
                    reinterpret_cast<int4*>(acc_s + w0)[i] = make_int4(0, 0, 0, 0);
            }
            __syncthreads();
        } else if (kind == kUnitUpdate) {
            update_chunk<STATS>(n, t, s_idx[b] * blockDim.x + tid, odd ? n.accx : n.acc0);
            if (tid == 0) take(atomicAdd(n.tile_ctr + (t & 1ull), 1u) + gridDim.x, b ^ 1u);
            __syncthreads();
        } else {  // the plan of the next step, in the accumulators' shared memory
            plan_step<kFusedThreads>(n, t + 1, F.tiles, F.n_tiles, odd ? F.plan[0] : F.plan[1], F.n_ctas, F.cap,
                                     F.items_cap, reinterpret_cast<unsigned char*>(acc_s));
            __syncthreads();
            for (uint32_t i = tid; i < (F.plan_bytes + 15u) / 16u; i += blockDim.x)
                reinterpret_cast<int4*>(acc_s)[i] = make_int4(0, 0, 0, 0);
            if (tid == 0) take(atomicAdd(n.tile_ctr + (t & 1ull), 1u) + gridDim.x, b ^ 1u);
            __syncthreads();
        }
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (lane == 0 && ev) atomicAdd(&n.ctl->events, ev);
    if (bad) atomicOr(&n.ctl->err, kErrBadTarget);
}

}  // namespace snn
