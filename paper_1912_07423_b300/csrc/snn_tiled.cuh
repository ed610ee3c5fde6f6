// snn_tiled.cuh -- Receive Spikes with the accumulators in shared memory.
//
// The paper delivers a spike with one CUDA block walking the spiker's
// adjacency row and updating the recipients with atomics (Section III-A-2).
// On a B300 the random 32-bit red.global.add that such a walk issues runs at
// about 2e11 per second into L2 (a fifth of what HBM can stream in edges),
// while shared-memory atomics run about five times faster.  This form keeps
// the walk over whole rows but adds into accumulators held in the CTA's
// shared memory:
//
//   * a network instance is a TILE when its accumulators fit one CTA's shared
//     memory; a larger instance is cut by target id into several tiles, and
//     the segment of a (sorted) row inside each tile comes from a split table
//     built once with the graph;
//   * every step a one-block kernel (k_plan) cuts the work of that step from
//     the spike counts of the step being delivered: tile k, with c_k arriving
//     spikes and w_k = c_k s_k expected work (s_k: mean row segment plus a
//     fixed cost per spike), gets P_k = ceil(w_k / target) spike parts,
//     target = sum(w) / (kItemsPerCta * CTAs); part p delivers spikes
//     [c_k p / P_k, c_k (p+1) / P_k).  The (tile, part) items are listed
//     heaviest first, and a persistent grid takes them one after the other
//     from an atomic counter;
//   * a part's copy of the accumulators leaves shared memory by one bulk
//     asynchronous copy (the TMA engine): a tile's only part copies it over
//     the global accumulators, the parts of a split tile add it into them
//     with the copy's element-wise integer reduction in L2 (the update left
//     them at zero).  Integer sums do not depend on the order of the adds.
//
// Every edge is read once per step, in whole coalesced rows; no global
// atomics are issued by the threads.  The plan follows each step's spikes,
// so a burst in one network is cut as finely as it needs; results do not
// depend on the plan, only the balance across SMs does.
//
// The bulk-copy kernel (snn_bulk.cuh) uses the same tiles with a static plan
// cut on the host from the expected or measured spike rates
// (TileDev::nparts, part_base; re-cut on the first steps).
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <functional>
#include <numeric>
#include <vector>

#include "../../include/snn.h"
#include "snn_device.cuh"

namespace snn {

struct TileDev {
    uint32_t inst;                  // instance
    uint32_t lo, len;               // padded id range [lo, lo + len); len is a multiple of 256
    uint32_t tau, ntiles;           // tile index inside the instance, tiles of the instance
    uint32_t nparts;                // static plan: spike parts of this tile
    uint32_t lpieces;               // per-step plan: a row segment is cut into 2^lpieces pieces
    uint32_t pbase;                 // the instance's first padded id
    float seg;                      // per-step plan: expected work per arriving spike (edges)
    uint32_t pad;
    unsigned long long split;       // base of the instance's split table: n_b rows x (ntiles-1) uint32
    unsigned long long part_base;   // static plan: base of the partials (nparts x CH x len int32) if nparts > 1
};

struct MergeDev {  // one chunk of a multi-part tile to add up
    uint32_t tile, off, len, pad;
};

// One work item of a step: spikes [s_beg, s_end) of tile k's instance, one of
// the tile's P parts.
struct ItemDev {
    uint32_t k, s_beg, s_end, P;
};

// The plan of one step, written by k_plan and read by the receive.
struct StepPlan {
    uint32_t* hdr = nullptr;   // [0] items
    ItemDev* items = nullptr;  // heaviest first
    uint32_t* parts = nullptr; // P_k (0: no spike arrives)
};

struct TiledPlan {
    TileDev* tiles = nullptr;
    uint32_t* split = nullptr;
    int32_t* partial = nullptr;
    // static plan (bulk-copy receive)
    uint32_t* items = nullptr;   // (tile << 8 | part), heaviest first
    MergeDev* merges = nullptr;
    uint32_t n_items = 0, n_merges = 0;
    // per-step plan (tiled receive)
    StepPlan step;
    bool dynamic = false;
    uint32_t n_tiles = 0;
    uint32_t max_len = 0;
    uint32_t grid = 0;
    uint32_t cap = 1;            // most parts of a tile in one step
    uint32_t items_cap = 0;      // per-step plan: room for items
    int channels = 1;
    int threads = 1024;
    size_t smem = 0;
};

// Two CTAs of 16 warps per SM, each with up to 112 KB of accumulators: while
// one waits at a barrier (its slowest warp, its copy-out), the other keeps
// the SM's loads in flight.
constexpr int kTiledThreads = 512;
constexpr int kTiledCtasPerSm = 2;
constexpr uint32_t kTiledMaxWords = 28672;  // int32 accumulators of one CTA (112 KB)
constexpr int kVec = 4;            // 4-edge vectors in flight per lane
constexpr uint32_t kMaxParts = 255;
constexpr uint32_t kMergeChunk = 4096;
constexpr int kPlanThreads = 1024;
constexpr uint32_t kPlanMaxTiles = 4096;
constexpr uint32_t kRankSortMax = 1024;  // most keys the rank sort's per-thread slots hold
constexpr uint32_t kRankSortUse = 128;   // up to this many tiles the plan sorts by rank, above by a bitonic network
constexpr float kItemsPerCta = 1.5f;     // per-step plan: items per CTA at the target size
constexpr float kSpikeCost = 8.0f;     // fixed work of one arriving spike, in edges
constexpr uint32_t kMaxLogPieces = 3;

// Edges are read once per step and never again before the rest of the
// (larger than L2) graph has streamed by, so their loads carry an L2
// evict-first policy: L2 keeps the partials, accumulators, queues and row
// records instead.
__device__ __forceinline__ unsigned long long evict_first_policy()
{
    unsigned long long p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint4 ld_edges4(const void* ptr, unsigned long long pol)
{
    uint4 v;
    asm("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint2 ld_edges2(const void* ptr, unsigned long long pol)
{
    uint2 v;
    asm("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint32_t ld_edge(const uint32_t* ptr, unsigned long long pol)
{
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
    return v;
}

__device__ __forceinline__ uint16_t ld_edge16(const int16_t* ptr, unsigned long long pol)
{
    uint16_t v;
    asm("ld.global.nc.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(v) : "l"(ptr), "l"(pol));
    return v;
}

// Edge layouts the receive reads: binary32 weights and u32 targets, int16
// weight codes and u32 targets, or one u32 per edge holding the target's
// offset in its instance (high half) and the int16 code (low half).
// kWOff16: every row carries one weight (the source population's, Table 2),
// held per row, and an edge is its target's 16-bit offset in its instance
// alone: 8 edges per 16-byte vector.
enum : int { kWF32 = 0, kW16 = 1, kWPacked = 2, kWOff16 = 3 };
__host__ __device__ constexpr int vec_of(int wm) { return wm == kWPacked ? 6 : (wm == kWOff16 ? 4 : kVec); }
__host__ __device__ constexpr uint32_t edge_bytes_of(int wm)
{
    return wm == kWF32 ? 8u : (wm == kW16 ? 6u : (wm == kWPacked ? 4u : 2u));
}

// ---------------------------------------------------------------------------
// Pipelined delivery of the spikes [s_beg, s_end) of the instance's queue q
// (local ids from pbase) to tile T.  The work is cut into units, piece
// u % K of the row segment of spike s_beg + u / K (K = 2^T.lpieces; the
// segment of a row inside the tile comes from the split table), strided
// over the warps.  A warp's units are walked as a stream of rounds -- up to PV 16-byte vectors per lane of one unit, plus
// its unaligned head and tail edges in its first round -- and the edge loads
// of the next round (of the same unit or the next one) are issued before the
// shared-memory atomics of the current round, so the load latency of one
// round runs under the atomics of the other and consecutive units follow
// each other without a gap.  The record of the next unit and the spike of
// the one after are loaded when a unit's first round is formed.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int pipe_vec_of(int wm) { return wm == kWPacked ? 3 : (wm == kWOff16 ? 2 : (wm == kW16 ? 2 : 1)); }
__host__ __device__ constexpr uint32_t pipe_epv_of(int wm) { return wm == kWOff16 ? 8u : 4u; }  // edges per vector

template <int WM>
struct PipeRound {
    static constexpr int PV = pipe_vec_of(WM);
    uint4 tv[PV];                              // targets, or packed edges
    uint2 wh[WM == kW16 ? PV : 1];             // int16 codes
    uint4 wf[WM == kWF32 ? PV : 1];            // binary32 weights
    uint32_t nv;                               // vectors of this lane in the round
    uint32_t sc;                               // shift | channel << 5 | head edge present << 6
    uint32_t hx, hw;                           // head / tail edge: raw target (or packed edge), raw weight
    int32_t rw;                                // kWOff16: the row's weight
};

template <int WM, int CH>
__device__ __forceinline__ void deliver_pipe(const Net& n, const TileDev& T, const uint32_t* q, uint32_t pbase,
                                             const uint32_t* sp, int32_t* acc_s, uint32_t s_beg, uint32_t s_end,
                                             unsigned long long pol, unsigned long long& ev, bool& bad)
{
    constexpr int PV = pipe_vec_of(WM);
    constexpr uint32_t EPV = pipe_epv_of(WM), RB = 32u * EPV;  // edges per vector, per warp vector row
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t nsplit = T.ntiles - 1, lk = T.lpieces;
    const uint32_t u_end = (s_end - s_beg) << lk;
    const uint32_t x0 = (WM == kWPacked || WM == kWOff16) ? T.lo - T.pbase : T.lo, tlen = T.len, tau = T.tau;
    // the next unit to form: u, its record (r, ylo, yhi, its weight rwn); the spike of unit u + nwarps: jn
    uint32_t u = warp, jn = 0, ylo = 0, yhi = 0;
    int32_t rwn = 0;
    uint4 r = make_uint4(0, 0, 0, 0);
    auto fetch = [&](uint32_t j) {
        r = __ldg(n.rinfo + j);
        if constexpr (WM == kWOff16) rwn = __ldg(n.roww + j);
        ylo = 0;
        yhi = 0xffffffffu;
        if (nsplit) {
            const uint32_t* sj = sp + (size_t)(j - pbase) * nsplit;
            if (tau > 0) ylo = __ldg(sj + tau - 1);
            if (tau < nsplit) yhi = __ldg(sj + tau);
        }
    };
    if (u < u_end) fetch(q[s_beg + (u >> lk)]);
    if (u + nwarps < u_end) jn = q[s_beg + ((u + nwarps) >> lk)];
    // the unit whose rounds are being formed: aligned vectors [cb, ce), first
    // round pending with its head / tail edges [pb, a4) and [b4, pe)
    uint64_t cb = 0, ce = 0, pb = 0, pe = 0;
    uint32_t csc = 0;
    int32_t crw = 0;
    bool first = false;
    // forms the next round into R and issues its loads; false when the warp's units are done
    auto issue = [&](PipeRound<WM>& R) -> bool {
        while (!first && cb >= ce) {  // the current unit is done: take the next non-empty one
            if (u >= u_end) return false;
            const uint64_t beg = ((unsigned long long)r.y << 32) | r.x;
            const uint64_t sb = beg + ylo, se = beg + (yhi == 0xffffffffu ? r.z : yhi);
            const uint64_t len = se - sb, c = u & ((1u << lk) - 1u);
            pb = sb + ((len * c) >> lk);
            pe = sb + ((len * (c + 1)) >> lk);
            csc = (r.w & 31u) | ((CH == 2 && (r.w & 0x80u)) ? 32u : 0u);
            crw = rwn;
            ev += pe - pb;
            // prefetch: the record of the unit after this one and the spike of the one after that
            const uint32_t u1 = u + nwarps;
            if (u1 < u_end) fetch(jn);
            if (u1 + nwarps < u_end) jn = q[s_beg + ((u1 + nwarps) >> lk)];
            u = u1;
            const uint64_t upa = (pb + EPV - 1) & ~(uint64_t)(EPV - 1), dna = pe & ~(uint64_t)(EPV - 1);
            cb = upa < pe ? upa : pe;
            ce = dna > cb ? dna : cb;
            first = pe > pb;
        }
        // this lane's vectors of the round: cb + EPV lane + RB i < ce
        const uint64_t rem = ce - cb;
        uint32_t nv = 0;
        if (rem > (uint64_t)EPV * lane) {
            const uint64_t k = (rem - (uint64_t)EPV * lane + RB - 1) / RB;
            nv = k < (uint64_t)PV ? (uint32_t)k : (uint32_t)PV;
        }
        R.nv = nv;
        R.sc = csc;
        R.rw = crw;
#pragma unroll
        for (int i = 0; i < PV; ++i) {
            const uint64_t e = cb + (uint64_t)EPV * lane + (uint64_t)RB * i;
            if ((uint32_t)i < nv) {
                if constexpr (WM == kWPacked) {
                    R.tv[i] = ld_edges4(n.pk + e, pol);
                } else if constexpr (WM == kWOff16) {
                    R.tv[i] = ld_edges4(n.pk16 + e, pol);
                } else {
                    R.tv[i] = ld_edges4(n.tgt + e, pol);
                    if constexpr (WM == kW16) R.wh[i] = ld_edges2(n.w16 + e, pol);
                    else R.wf[i] = ld_edges4(n.w32 + e, pol);
                }
            }
        }
        if (first) {  // the unaligned head [pb, cb) on lanes 0..EPV-1, tail [ce, pe) on lanes EPV..2 EPV-1
            uint64_t e = ~0ull;
            if (lane < cb - pb)
                e = pb + lane;
            else if (lane >= EPV && lane - EPV < pe - ce)
                e = ce + (lane - EPV);
            if (e != ~0ull) {
                R.sc |= 64u;
                if constexpr (WM == kWPacked) {
                    R.hx = ld_edge(n.pk + e, pol);
                } else if constexpr (WM == kWOff16) {
                    R.hx = ld_edge16(reinterpret_cast<const int16_t*>(n.pk16 + e), pol);
                } else {
                    R.hx = ld_edge(n.tgt + e, pol);
                    if constexpr (WM == kW16) R.hw = ld_edge16(n.w16 + e, pol);
                    else R.hw = ld_edge(reinterpret_cast<const uint32_t*>(n.w32 + e), pol);
                }
            }
            first = false;
        }
        cb += (uint64_t)RB * PV;
        if (cb > ce) cb = ce;
        return true;
    };
    auto add = [&](int32_t* a, uint32_t x, int32_t w) {
        if (x < tlen)
            atomicAdd(a + x, w);
        else
            bad = true;
    };
    auto process = [&](const PipeRound<WM>& R) {
        const uint32_t shift = R.sc & 31u;
        int32_t* a = acc_s + ((CH == 2 && (R.sc & 32u)) ? tlen : 0u);
#pragma unroll
        for (int i = 0; i < PV; ++i) {
            if ((uint32_t)i >= R.nv) continue;
            const uint32_t v[4] = {R.tv[i].x, R.tv[i].y, R.tv[i].z, R.tv[i].w};
            if constexpr (WM == kWOff16) {
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    add(a, (v[k] & 0xffffu) - x0, R.rw);
                    add(a, (v[k] >> 16) - x0, R.rw);
                }
                continue;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if constexpr (WM == kWPacked) {
                    add(a, (v[k] >> 16) - x0, (int32_t)(int16_t)(v[k] & 0xffffu) << shift);
                } else if constexpr (WM == kW16) {
                    const uint32_t h2 = k < 2 ? R.wh[i].x : R.wh[i].y;
                    add(a, v[k] - x0, (int32_t)(int16_t)((k & 1) ? (h2 >> 16) : (h2 & 0xffffu)) << shift);
                } else {
                    const uint32_t f = k == 0 ? R.wf[i].x : k == 1 ? R.wf[i].y : k == 2 ? R.wf[i].z : R.wf[i].w;
                    add(a, v[k] - x0, __float2int_rz(__uint_as_float(f)));
                }
            }
        }
        if (R.sc & 64u) {
            if constexpr (WM == kWOff16)
                add(a, (R.hx & 0xffffu) - x0, R.rw);
            else if constexpr (WM == kWPacked)
                add(a, (R.hx >> 16) - x0, (int32_t)(int16_t)(R.hx & 0xffffu) << shift);
            else if constexpr (WM == kW16)
                add(a, R.hx - x0, (int32_t)(int16_t)(R.hw & 0xffffu) << shift);
            else
                add(a, R.hx - x0, __float2int_rz(__uint_as_float(R.hw)));
        }
    };
    PipeRound<WM> A, B;
    bool hA = issue(A);
    while (hA) {
        const bool hB = issue(B);
        process(A);
        if (!hB) break;
        hA = issue(A);
        process(B);
    }
}

// Shared memory of k_plan for n_pad (a power of two >= the tiles) entries.
__host__ __device__ inline size_t plan_smem(uint32_t n_pad) { return (size_t)n_pad * 20; }

// The plan of step t's receive (one block of PT threads; plan_s: plan_smem
// bytes of shared memory).  Tile k gets P_k parts as the header of this file
// states; the items are ordered by work per part, heaviest first, ties by
// tile index: 64-bit keys sorted by rank (each key counts the smaller ones)
// or, for many tiles, by a bitonic network.
template <int PT>
__device__ __forceinline__ void plan_step(const Net& n, unsigned long long t, const TileDev* __restrict__ tiles,
                                          uint32_t n_tiles, const StepPlan& sp, uint32_t n_ctas, uint32_t cap,
                                          uint32_t items_cap, unsigned char* plan_s)
{
    static_assert(PT >= 32 && PT % 32 == 0 && kRankSortMax % PT == 0, "whole warps, rank-sort slots per thread");
    __shared__ float red[PT / 32];
    __shared__ uint32_t s_act, s_items;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (t + 1 < n.d) {
        if (threadIdx.x == 0) sp.hdr[0] = 0;
        return;
    }
    uint32_t n_pad = 1;
    while (n_pad < n_tiles) n_pad <<= 1;
    unsigned long long* key = reinterpret_cast<unsigned long long*>(plan_s);  // later: item offset by position
    uint32_t* pk = reinterpret_cast<uint32_t*>(key + n_pad);                 // spikes, then P_k
    float* wk = reinterpret_cast<float*>(pk + n_pad);                        // later: rank, then tile by position
    uint32_t* at = reinterpret_cast<uint32_t*>(wk);
    uint32_t* ck = reinterpret_cast<uint32_t*>(wk + n_pad);                  // spikes
    uint32_t* off = reinterpret_cast<uint32_t*>(key);
    if (threadIdx.x == 0) s_act = 0;
    const unsigned long long ts = t + 1 - n.d;
    const uint32_t* cnt = n.icount + (size_t)(ts & (n.cr - 1)) * n.n_inst;
    float wsum = 0.f;
    for (uint32_t k = threadIdx.x; k < n_tiles; k += blockDim.x) {
        const uint32_t c = cnt[__ldg(&tiles[k].inst)];
        const float w = (float)c * __ldg(&tiles[k].seg);
        pk[k] = c;
        ck[k] = c;
        wk[k] = w;
        wsum += w;
    }
    for (int o = 16; o; o >>= 1) wsum += __shfl_xor_sync(0xffffffffu, wsum, o);
    if (lane == 0) red[warp] = wsum;
    __syncthreads();
    float W = 0.f;
    for (uint32_t i = 0; i < PT / 32; ++i) W += red[i];
    const float target = W / (kItemsPerCta * (float)n_ctas);
    for (uint32_t k = threadIdx.x; k < n_pad; k += blockDim.x) {
        unsigned long long kk = ~0ull;
        if (k < n_tiles) {
            const uint32_t c = pk[k];
            uint32_t P = 0;
            if (c) {
                P = 1;
                if (target > 0.f) {
                    const float x = ceilf(wk[k] / target);
                    P = x < (float)cap ? (x > 1.f ? (uint32_t)x : 1u) : cap;
                }
                P = P < c ? P : c;
                kk = ((unsigned long long)(~__float_as_uint(wk[k] / (float)P)) << 32) | k;
                atomicAdd(&s_act, 1u);
            }
            pk[k] = P;
            sp.parts[k] = P;
        }
        key[k] = kk;
    }
    __syncthreads();
    const uint32_t n_act = s_act;  // the active keys sort first
    if (n_pad <= kRankSortUse) {
        // rank of key k = keys below it; g threads per key, each over n_pad / g keys
        uint32_t* rank = at;
        for (uint32_t k = threadIdx.x; k < n_pad; k += blockDim.x) rank[k] = 0;
        __syncthreads();
        uint32_t g = n_pad >= blockDim.x ? 1u : blockDim.x / n_pad;  // a power of two
        g = g < n_pad ? g : n_pad;  // at least one key per thread
        const uint32_t span = n_pad / g;
        for (uint32_t idx = threadIdx.x; idx < n_pad * g; idx += blockDim.x) {
            const uint32_t k = idx / g, j0 = (idx % g) * span;
            const unsigned long long kk = key[k];
            if (kk == ~0ull) continue;
            uint32_t c = 0;
            for (uint32_t j = j0; j < j0 + span; ++j) c += key[j] < kk ? 1u : 0u;
            if (c) atomicAdd(&rank[k], c);
        }
        __syncthreads();
        uint32_t r[kRankSortMax / PT];
        for (uint32_t i = 0, k = threadIdx.x; i < kRankSortMax / PT; ++i, k += blockDim.x)
            r[i] = (k < n_pad && key[k] != ~0ull) ? rank[k] : ~0u;
        __syncthreads();
        for (uint32_t i = 0, k = threadIdx.x; i < kRankSortMax / PT; ++i, k += blockDim.x)
            if (r[i] != ~0u) at[r[i]] = k;
    } else {
        for (uint32_t size = 2; size <= n_pad; size <<= 1) {
            for (uint32_t stride = size >> 1; stride; stride >>= 1) {
                for (uint32_t i = threadIdx.x; i < n_pad / 2; i += blockDim.x) {
                    const uint32_t lo = 2 * i - (i & (stride - 1)), hi = lo + stride;
                    const unsigned long long a = key[lo], b = key[hi];
                    if ((a > b) == ((lo & size) == 0)) {
                        key[lo] = b;
                        key[hi] = a;
                    }
                }
                __syncthreads();
            }
        }
        for (uint32_t pos = threadIdx.x; pos < n_act; pos += blockDim.x) at[pos] = (uint32_t)key[pos];
    }
    __syncthreads();
    // warp 0: item offsets by position; lane l takes positions [l m, (l+1) m)
    if (warp == 0) {
        const uint32_t m = (n_act + 31) / 32;
        const uint32_t beg = lane * m < n_act ? lane * m : n_act, end = beg + m < n_act ? beg + m : n_act;
        uint32_t ni = 0;
        for (uint32_t pos = beg; pos < end; ++pos) ni += pk[at[pos]];
        uint32_t x = ni;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
        uint32_t o = x - ni;
        for (uint32_t pos = beg; pos < end; ++pos) {
            off[pos] = o;
            o += pk[at[pos]];
        }
        if (lane == 31) {
            const bool fits = x <= items_cap;
            if (!fits) atomicOr(&n.ctl->err, kErrPlan);
            s_items = fits ? x : 0u;
            sp.hdr[0] = fits ? x : 0u;
        }
    }
    __syncthreads();
    // every thread: item i belongs to the last position whose offset is <= i
    const uint32_t n_items = s_items;
    for (uint32_t i = threadIdx.x; i < n_items; i += blockDim.x) {
        uint32_t lo = 0, hi = n_act;  // off[lo] <= i < off[hi] (off[n_act] = n_items)
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (off[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        const uint32_t k = at[lo], part = i - off[lo], P = pk[k], c = ck[k];
        sp.items[i] = ItemDev{k, (uint32_t)((unsigned long long)c * part / P),
                              (uint32_t)((unsigned long long)c * (part + 1) / P), P};
    }
}

// The plan of the launch's step as a kernel of its own (one block).
__global__ void __launch_bounds__(kPlanThreads, 1) k_plan(Net n, const TileDev* __restrict__ tiles, uint32_t n_tiles,
                                                          StepPlan sp, uint32_t n_ctas, uint32_t cap, uint32_t items_cap)
{
    extern __shared__ __align__(16) unsigned char plan_s[];
    plan_step<kPlanThreads>(n, n.ctl->t + n.k, tiles, n_tiles, sp, n_ctas, cap, items_cap, plan_s);
}

// Issues the bulk copy of bytes of shared memory s to global memory g, as a
// plain copy or an element-wise int32 add into g.  Both addresses 16-byte
// aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_out(int32_t* g, const int32_t* s, uint32_t bytes, bool add)
{
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(s);
    if (add)
        asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.s32 [%0], [%1], %2;"
                     ::"l"(g), "r"(sa), "r"(bytes) : "memory");
    else
        asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(g), "r"(sa), "r"(bytes)
                     : "memory");
}

// The receive of one step under the per-step plan.  CTA c starts with item c
// and takes the next ones from an atomic counter; thread 0 takes and reads
// the CTA's next item when it is done with its own units of the current
// one, while the other warps finish theirs.  With pdl set the kernel was
// launched while the step's update may still run (programmatic dependent
// launch): it reads nothing the update writes, and waits for the update to
// finish before its first copy into the accumulators, which the update
// reads and clears.
template <int WM, int CH>
__global__ void __launch_bounds__(kTiledThreads, kTiledCtasPerSm) k_receive_tiled(Net n, const TileDev* __restrict__ tiles,
                                                                    uint32_t n_tiles, StepPlan sp,
                                                                    const uint32_t* __restrict__ split, uint32_t max_len,
                                                                    uint32_t pdl)
{
    extern __shared__ __align__(16) int32_t acc_s[];  // CH * max_len (the current tile uses CH * len)
    __shared__ TileDev s_T[2];
    __shared__ ItemDev s_I[2];
    __shared__ uint32_t s_ok[2];
    const unsigned long long t = n.ctl->t + n.k;
    const uint32_t lane = threadIdx.x & 31u;
    unsigned int* ctr = n.tile_ctr + (t & 1ull);
    const uint32_t n_items = sp.hdr[0];
    const unsigned long long ts = t + 1 >= n.d ? t + 1 - n.d : 0ull;
    unsigned long long ev = 0;  // every lane of a warp counts the warp's segments; lane 0 reports
    bool bad = false;           // a target outside the tile: the split table does not match the rows
    if (blockIdx.x >= n_items) return;
    const unsigned long long pol = evict_first_policy();
    const uint32_t* qs = n.q + (size_t)(ts % n.D) * n.Np;
    // item it's record and tile into buffer b (thread 0); false when the plan is done
    auto take = [&](uint32_t it, uint32_t b) {
        bool ok = it < n_items;
        if (ok) {
            const ItemDev I = sp.items[it];
            if (I.k < n_tiles && I.s_beg <= I.s_end) {
                s_I[b] = I;
                s_T[b] = tiles[I.k];
            } else {  // not produced by a correct plan: report, touch nothing
                atomicOr(&n.ctl->err, kErrPlan);
                ok = false;
            }
        }
        s_ok[b] = ok ? 1u : 0u;
    };
    if (threadIdx.x == 0) take(blockIdx.x, 0);
    // the accumulators start at zero, and every item leaves them at zero
    for (uint32_t i = threadIdx.x; i < CH * max_len / 4; i += blockDim.x)
        reinterpret_cast<int4*>(acc_s)[i] = make_int4(0, 0, 0, 0);
    __syncthreads();
    for (uint32_t b = 0; s_ok[b]; b ^= 1u) {
        const ItemDev& I = s_I[b];  // read from shared memory where used
        const TileDev& T = s_T[b];
        deliver_pipe<WM, CH>(n, T, qs + T.pbase, T.pbase, split + T.split, acc_s, I.s_beg, I.s_end, pol, ev, bad);
        if (threadIdx.x == 0) take(atomicAdd(ctr, 1u) + gridDim.x, b ^ 1u);
        // the tile's pending input for the next update, or this part's share
        // of it: the shared-memory adds are made visible to the copy engine,
        // which reads them out before they are cleared
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        // the CTA's last item (no next one taken): its accumulators need no
        // clearing, and the copy is waited for once, before the CTA exits
        {  // warp w copies out and clears slice w of the CH * len words (1/16 of a
           // channel or more: slices are multiples of 16 words, inside one channel)
            const uint32_t nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5;
            const uint32_t per = CH * T.len / nwarps, w0 = warp * per;
            if (lane == 0) {
                if (pdl) {  // the update before this kernel reads and clears the accumulators: wait for it
                    asm volatile("griddepcontrol.wait;" ::: "memory");
                    pdl = 0;
                }
                const uint32_t ch = CH == 2 && w0 >= T.len ? 1u : 0u;
                bulk_out((ch ? n.acc1 : n.acc0) + T.lo + (w0 - ch * T.len), acc_s + w0, per * 4u, I.P > 1);
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                if (s_ok[b ^ 1u]) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
            }
            if (s_ok[b ^ 1u]) {
                __syncwarp();
                for (uint32_t i = lane; i < per / 4; i += 32)
                    reinterpret_cast<int4*>(acc_s + w0)[i] = make_int4(0, 0, 0, 0);
            }
        }
        __syncthreads();
    }
    if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    if (lane == 0 && ev) atomicAdd(&n.ctl->events, ev);
    if (bad) atomicOr(&n.ctl->err, kErrBadTarget);
}

// Adds up the partials of chunk of a multi-part tile: one int4 per thread,
// eight partials' loads in flight.
template <int CH>
__device__ __forceinline__ void merge_chunk(const Net& n, const TileDev& T, const MergeDev& M, const int32_t* base,
                                            uint32_t nparts)
{
    const uint32_t i = M.off + threadIdx.x * 4;
    if (i >= M.off + M.len) return;
    for (uint32_t c = 0; c < CH; ++c) {
        const int32_t* src = base + (size_t)c * T.len + i;
        const size_t stride = (size_t)CH * T.len;  // between parts
        int4 s = make_int4(0, 0, 0, 0);
        uint32_t p = 0;
        for (; p + 8 <= nparts; p += 8) {
            int4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = __ldg(reinterpret_cast<const int4*>(src + (p + u) * stride));
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                s.x += v[u].x;
                s.y += v[u].y;
                s.z += v[u].z;
                s.w += v[u].w;
            }
        }
        for (; p < nparts; ++p) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(src + p * stride));
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        *reinterpret_cast<int4*>((c ? n.acc1 : n.acc0) + T.lo + i) = s;
    }
}

// Static plan: one chunk per block.
template <int CH>
__global__ void __launch_bounds__(kMergeChunk / 4) k_merge_parts(Net n, const TileDev* __restrict__ tiles,
                                                                const MergeDev* __restrict__ merges,
                                                                const int32_t* __restrict__ partial)
{
    const MergeDev M = merges[blockIdx.x];
    const TileDev T = tiles[M.tile];
    const unsigned long long t = n.ctl->t + n.k;
    if (t + 1 < n.d) return;
    const unsigned long long ts = t + 1 - n.d;
    if (n.icount[(size_t)(ts & (n.cr - 1)) * n.n_inst + T.inst] == 0) return;  // no part wrote anything
    merge_chunk<CH>(n, T, M, partial + T.part_base, T.nparts);
}

// Split table of one multi-tile instance: for local row l and inner boundary
// tau (1..ntiles-1), the offset inside the row of the first target >= the
// boundary's padded id, stored at [l * (ntiles-1) + tau - 1].
__global__ void k_split_rows(const uint64_t* roff, const uint32_t* tgt, uint32_t pbase, uint32_t nb,
                             const uint32_t* bounds /* ntiles+1 padded ids */, uint32_t ntiles, uint32_t* split)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t l = warp; l < nb; l += nwarps) {
        const uint64_t beg = roff[pbase + l], end = roff[pbase + l + 1];
        for (uint32_t tau = 1 + lane; tau < ntiles; tau += 32) {
            const uint32_t v = bounds[tau];
            uint64_t lo = beg, hi = end;
            while (lo < hi) {
                const uint64_t mid = (lo + hi) >> 1;
                if (tgt[mid] < v)
                    lo = mid + 1;
                else
                    hi = mid;
            }
            split[(size_t)l * (ntiles - 1) + (tau - 1)] = (uint32_t)(lo - beg);
        }
    }
}

inline cudaError_t tiled_set_smem(size_t smem)
{
    cudaError_t e = cudaSuccess;
    const int s = (int)smem;
    const auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWF32, 1>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kW16, 1>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWPacked, 1>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWF32, 2>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kW16, 2>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWPacked, 2>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWOff16, 1>, attr, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<kWOff16, 2>, attr, s);
    return e;
}

inline void tiled_free(TiledPlan& P, const std::function<void(void*)>& release)
{
    release(P.tiles);
    release(P.split);
    release(P.partial);
    release(P.items);
    release(P.merges);
    release(P.step.hdr);
    release(P.step.items);
    release(P.step.parts);
    P = TiledPlan{};
}

// Build the tiles and, for the bulk-copy receive (dynamic false), its static
// plan.  An instance is cut by target into tiles of at most max_len padded
// ids (the shared-memory limit).  Static plan: work[b] is the expected
// delivered edges of instance b per step (any positive scale; null:
// proportional to its synapses); with target = total / (1.25 CTAs) a tile of
// expected work w gets ceil(w / target) spike parts.  Per-step plan (dynamic
// true): the buffers k_plan fills, sized for the most it can write --
// sum_k P_k <= kItemsPerCta CTAs + tiles, since P_k <= w_k / target + 1, and
// likewise for the partial words.  Needs sorted rows when an instance has
// several tiles.  A tile's row segments are cut into 2^lpieces pieces only
// where the mean segment reaches 1.5 piece_edges (and again at each doubling),
// so that every unit keeps a warp busy for a few rounds of loads.
inline snn_status tiled_plan(TiledPlan& P, const Net& n, const snn_params* params, const uint32_t* pbase,
                             uint32_t n_inst, int channels, uint32_t max_len, const double* work,
                             const uint64_t* inst_edges, int sms, const std::function<void*(size_t)>& alloc,
                             const std::function<void(void*)>& release, cudaStream_t s, bool dynamic,
                             uint32_t piece_edges)
{
    max_len = std::max<uint32_t>(256, max_len / 256 * 256);
    std::vector<double> wk(n_inst, 0.0);
    for (uint32_t b = 0; b < n_inst; ++b) wk[b] = work ? work[b] : (double)inst_edges[b];
    const double total = std::accumulate(wk.begin(), wk.end(), 0.0);

    std::vector<TileDev> tiles;
    std::vector<double> tile_work;
    std::vector<std::vector<uint32_t>> bounds(n_inst);
    std::vector<unsigned long long> split_base(n_inst, 0);
    unsigned long long split_total = 0;
    uint32_t longest = 0;
    for (uint32_t b = 0; b < n_inst; ++b) {
        const uint32_t npad = pbase[b + 1] - pbase[b];
        if (npad == 0) continue;
        const uint32_t m = npad / 256;
        const uint32_t T = std::min<uint32_t>((npad + max_len - 1) / max_len, m);
        auto& B = bounds[b];
        B.resize(T + 1);
        for (uint32_t tau = 0; tau <= T; ++tau) B[tau] = pbase[b] + 256u * (uint32_t)((unsigned long long)tau * m / T);
        split_base[b] = split_total;
        for (uint32_t tau = 0; tau < T; ++tau) {
            TileDev d{};
            d.inst = b;
            d.lo = B[tau];
            d.len = B[tau + 1] - B[tau];
            d.tau = tau;
            d.ntiles = T;
            d.nparts = 1;
            d.pbase = pbase[b];
            // mean segment of a row in this tile, plus the fixed cost of a spike
            const double mseg = params[b].n ? (double)inst_edges[b] / params[b].n * d.len / npad : 0.0;
            d.seg = (float)mseg + kSpikeCost;
            d.lpieces = 0;
            while (d.lpieces < kMaxLogPieces && mseg >= (double)(2u << d.lpieces) * piece_edges * 0.75) ++d.lpieces;
            d.split = split_base[b];
            tiles.push_back(d);
            tile_work.push_back(wk[b] * d.len / npad);
            longest = std::max(longest, d.len);
        }
        if (T > 1) split_total += (unsigned long long)(T - 1) * params[b].n;
    }
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const size_t smem = (size_t)longest * channels * 4;
    if (tiles.empty() || smem > (size_t)optin || tiles.size() >= (1u << 24)) return SNN_E_ARG;
    if (dynamic && tiles.size() > kPlanMaxTiles) return SNN_E_ARG;
    if (tiled_set_smem(smem) != cudaSuccess) return SNN_E_CUDA;
    int ctas = 0;
    cudaError_t oe = channels == 2
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_receive_tiled<kW16, 2>, kTiledThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_receive_tiled<kW16, 1>, kTiledThreads, smem);
    if (oe != cudaSuccess || ctas < 1) {
        cudaGetLastError();
        ctas = 1;
    }
    const uint32_t n_ctas = (uint32_t)(sms * ctas);
    const uint32_t cap = std::min<uint32_t>(kMaxParts, n_ctas);

    TiledPlan Q;
    Q.dynamic = dynamic;
    Q.n_tiles = (uint32_t)tiles.size();
    Q.max_len = longest;
    Q.channels = channels;
    Q.threads = kTiledThreads;
    Q.smem = smem;
    Q.cap = cap;
    std::vector<uint32_t> codes;
    std::vector<MergeDev> merges;
    unsigned long long part_total = 0;
    if (!dynamic) {  // static parts, heaviest first
        const double target = total > 0 ? total / (1.25 * n_ctas) : 1.0;
        struct Item {
            uint32_t code;
            double w;
        };
        std::vector<Item> items;
        for (uint32_t k = 0; k < tiles.size(); ++k) {
            TileDev& d = tiles[k];
            uint32_t parts = total > 0 ? (uint32_t)std::ceil(tile_work[k] / target) : 1u;
            parts = std::max<uint32_t>(1, std::min<uint32_t>(parts, cap));
            d.nparts = parts;
            if (parts > 1) {
                d.part_base = part_total;
                part_total += (unsigned long long)parts * channels * d.len;
                for (uint32_t off = 0; off < d.len; off += kMergeChunk)
                    merges.push_back(MergeDev{k, off, std::min(kMergeChunk, d.len - off), 0});
            }
            for (uint32_t p = 0; p < parts; ++p) items.push_back(Item{(k << 8) | p, tile_work[k] / parts});
        }
        std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.w > b.w; });
        for (const Item& it : items) codes.push_back(it.code);
        Q.n_items = (uint32_t)codes.size();
        Q.n_merges = (uint32_t)merges.size();
        Q.grid = std::min<uint32_t>(Q.n_items, n_ctas);
        Q.items = static_cast<uint32_t*>(alloc(codes.size() * 4));
        Q.merges = static_cast<MergeDev*>(alloc(std::max<size_t>(merges.size(), 1) * sizeof(MergeDev)));
    } else {
        // sum_k P_k <= sum_k (w_k / target + 1) = kItemsPerCta CTAs + tiles
        Q.items_cap = (uint32_t)std::ceil(kItemsPerCta * n_ctas) + 16 + (uint32_t)tiles.size();
        Q.grid = n_ctas;
        Q.step.hdr = static_cast<uint32_t*>(alloc(4 * sizeof(uint32_t)));
        Q.step.items = static_cast<ItemDev*>(alloc((size_t)Q.items_cap * sizeof(ItemDev)));
        Q.step.parts = static_cast<uint32_t*>(alloc(tiles.size() * 4));
        uint32_t n_pad = 1;
        while (n_pad < tiles.size()) n_pad <<= 1;
        if (cudaFuncSetAttribute(k_plan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan_smem(n_pad)) !=
            cudaSuccess)
            return SNN_E_CUDA;
    }
    Q.tiles = static_cast<TileDev*>(alloc(tiles.size() * sizeof(TileDev)));
    Q.split = static_cast<uint32_t*>(alloc(std::max<unsigned long long>(split_total, 1) * 4));
    Q.partial = static_cast<int32_t*>(alloc(std::max<unsigned long long>(part_total, 4) * 4));
    uint32_t* dbounds = static_cast<uint32_t*>(alloc(65536 * 4));
    const bool have = dynamic ? (Q.step.hdr && Q.step.items && Q.step.parts) : (Q.items && Q.merges);
    snn_status st = (have && Q.tiles && Q.split && Q.partial && dbounds) ? SNN_OK : SNN_E_NOMEM;
    if (st == SNN_OK &&
        (cudaMemcpyAsync(Q.tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         (dynamic && cudaMemsetAsync(Q.step.hdr, 0, 4 * sizeof(uint32_t), s) != cudaSuccess) ||
         (codes.size() && cudaMemcpyAsync(Q.items, codes.data(), codes.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) ||
         (merges.size() && cudaMemcpyAsync(Q.merges, merges.data(), merges.size() * sizeof(MergeDev),
                                           cudaMemcpyHostToDevice, s) != cudaSuccess)))
        st = SNN_E_CUDA;
    for (uint32_t b = 0; b < n_inst && st == SNN_OK; ++b) {
        const auto& B = bounds[b];
        if (B.size() <= 2) continue;
        const uint32_t T = (uint32_t)B.size() - 1;
        if (T + 1 > 65536) {
            st = SNN_E_ARG;
            break;
        }
        if (cudaMemcpyAsync(dbounds, B.data(), B.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) {
            st = SNN_E_CUDA;
            break;
        }
        k_split_rows<<<1184, 256, 0, s>>>(n.roff, n.tgt, pbase[b], params[b].n, dbounds, T, Q.split + split_base[b]);
        if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess) st = SNN_E_CUDA;
    }
    cudaStreamSynchronize(s);
    release(dbounds);
    if (st != SNN_OK) {
        tiled_free(Q, release);
        return st;
    }
    tiled_free(P, release);
    P = Q;
    return SNN_OK;
}

// The per-step plan of one step.
inline cudaError_t enqueue_tiled_plan(const TiledPlan& P, const Net& n, cudaStream_t s, int priority = 0)
{
    uint32_t n_pad = 1;
    while (n_pad < P.n_tiles) n_pad <<= 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(1);
    cfg.blockDim = dim3(kPlanThreads);
    cfg.dynamicSmemBytes = plan_smem(n_pad);
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = priority;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_plan, n, (const TileDev*)P.tiles, P.n_tiles, P.step, P.grid, P.cap, P.items_cap);
}

// The receive of one step under its plan; wm: the edge layout to read; pdl:
// launch it as a programmatic dependent of the kernel before it on s.
inline cudaError_t enqueue_tiled_receive(const TiledPlan& P, const Net& n, int wm, cudaStream_t s, bool pdl = false)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(P.grid);
    cfg.blockDim = dim3(P.threads);
    cfg.dynamicSmemBytes = P.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    const uint32_t flag = pdl ? 1u : 0u;
    auto go = [&](auto kernel) {
        return cudaLaunchKernelEx(&cfg, kernel, n, (const TileDev*)P.tiles, P.n_tiles, P.step, (const uint32_t*)P.split,
                                  P.max_len, flag);
    };
    if (P.channels == 2)
        return wm == kWOff16 ? go(k_receive_tiled<kWOff16, 2>)
               : wm == kWPacked ? go(k_receive_tiled<kWPacked, 2>)
               : wm == kW16     ? go(k_receive_tiled<kW16, 2>)
                                : go(k_receive_tiled<kWF32, 2>);
    return wm == kWOff16 ? go(k_receive_tiled<kWOff16, 1>)
           : wm == kWPacked ? go(k_receive_tiled<kWPacked, 1>)
           : wm == kW16     ? go(k_receive_tiled<kW16, 1>)
                            : go(k_receive_tiled<kWF32, 1>);
}

// 16-bit offsets (kWOff16) of every row's targets in their instance.
__global__ void k_pack_off16(Net n, uint32_t Np, uint16_t* pk16)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint32_t pb = n.inst[n.inst_of_w32[pj >> 5]].pbase;
        const uint64_t beg = n.roff[pj], end = n.roff[pj + 1];
        for (uint64_t e = beg + lane; e < end; e += 32) pk16[e] = (uint16_t)(n.tgt[e] - pb);
    }
}

// Packed edges (kWPacked) of every row: (target - instance base) << 16 | code.
__global__ void k_pack_edges(Net n, uint32_t Np, uint32_t* pk)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
    for (uint32_t pj = warp; pj < Np; pj += nwarps) {
        const uint32_t pb = n.inst[n.inst_of_w32[pj >> 5]].pbase;
        const uint64_t beg = n.roff[pj], end = n.roff[pj + 1];
        for (uint64_t e = beg + lane; e < end; e += 32)
            pk[e] = ((n.tgt[e] - pb) << 16) | (uint16_t)n.w16[e];
    }
}

}  // namespace snn
