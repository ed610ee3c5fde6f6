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
//   * a tile whose expected work is large is split by SPIKES into P parts:
//     part p delivers its share of the instance's spikes into a private copy
//     of the tile's accumulators.  A part that is alone stores its copy to the
//     global accumulators; otherwise it stores it to a partial buffer, and a
//     second kernel adds the P partials up (coalesced, L2-resident).
//
// Every edge is read once per step, in whole coalesced rows; no global
// atomics are issued.  The (tile, part) work items are listed heaviest first
// and a persistent grid takes them one after the other from an atomic
// counter.  Expected work comes from the edges at first and from the spike
// counts measured on the first steps after the one-time re-plan; results do
// not depend on the plan, only the balance across SMs does.
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
    uint32_t nparts;                // spike parts of this tile
    unsigned long long split;       // base of the instance's split table: n_b rows x (ntiles-1) uint32
    unsigned long long part_base;   // base of the tile's partials (nparts x len int32) if nparts > 1
};

struct MergeDev {  // one chunk of a multi-part tile to add up
    uint32_t tile, off, len, pad;
};

struct TiledPlan {
    TileDev* tiles = nullptr;
    uint32_t* items = nullptr;   // (tile << 8 | part), heaviest first
    uint32_t* split = nullptr;
    int32_t* partial = nullptr;
    MergeDev* merges = nullptr;
    uint32_t n_tiles = 0, n_items = 0, n_merges = 0;
    uint32_t max_len = 0;
    uint32_t grid = 0;
    int channels = 1;
    int threads = 1024;
    size_t smem = 0;
};

constexpr int kTiledThreads = 1024;
constexpr int kVec = 4;            // 4-edge vectors in flight per lane
constexpr uint32_t kMaxParts = 255;
constexpr uint32_t kMergeChunk = 4096;

template <bool W16>
__device__ __forceinline__ int32_t weight_at(const Net& n, uint64_t e, uint32_t shift)
{
    return W16 ? ((int32_t)__ldg(n.w16 + e) << shift) : __float2int_rz(__ldg(n.w32 + e));
}

template <bool W16, int CH>
__global__ void __launch_bounds__(kTiledThreads, 1) k_receive_tiled(Net n, const TileDev* __restrict__ tiles,
                                                                    const uint32_t* __restrict__ items,
                                                                    const uint32_t* __restrict__ split,
                                                                    int32_t* __restrict__ partial, uint32_t n_items,
                                                                    uint32_t max_len)
{
    extern __shared__ __align__(16) int32_t acc_s[];  // CH * max_len (the current tile uses CH * len)
    __shared__ uint32_t s_item;
    const unsigned long long t = n.ctl->t + n.k;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned int* ctr = n.tile_ctr + (t & 1ull);
    const bool deliver = t + 1 >= n.d;
    const unsigned long long ts = deliver ? t + 1 - n.d : 0ull;
    unsigned long long ev = 0;  // every lane of a warp counts the warp's segments; lane 0 reports
    bool bad = false;           // a target outside the tile: the split table does not match the rows
    // the accumulators start at zero, and every write-out leaves them at zero
    for (uint32_t i = threadIdx.x; i < CH * max_len / 4; i += blockDim.x)
        reinterpret_cast<int4*>(acc_s)[i] = make_int4(0, 0, 0, 0);
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items) break;
        const uint32_t code = __ldg(items + item);
        const TileDev T = tiles[code >> 8];
        const uint32_t part = code & 0xffu;
        const uint32_t cnt = deliver ? n.icount[(size_t)(ts & (n.cr - 1)) * n.n_inst + T.inst] : 0u;
        if (cnt == 0) {  // nothing arrives: the update already cleared these accumulators
            __syncthreads();
            continue;
        }
        const uint32_t pbase = __ldg(&n.inst[T.inst].pbase);
        const uint32_t* q = n.q + (size_t)(ts % n.D) * n.Np + pbase;
        const uint32_t nsplit = T.ntiles - 1;
        const uint32_t* sp = split + T.split;
        const uint32_t s_beg = (uint32_t)((unsigned long long)cnt * part / T.nparts);
        const uint32_t s_end = (uint32_t)((unsigned long long)cnt * (part + 1) / T.nparts);
        // one spike per warp; the next spike's row record is fetched while
        // the current row is delivered
        uint32_t s = s_beg + warp;
        uint32_t j = 0;
        uint4 r = make_uint4(0, 0, 0, 0);
        if (s < s_end) {
            j = q[s];
            r = __ldg(n.rinfo + j);
        }
        while (s < s_end) {
            const uint32_t s_next = s + nwarps;
            uint32_t j_next = 0;
            uint4 r_next = make_uint4(0, 0, 0, 0);
            if (s_next < s_end) {
                j_next = q[s_next];
                r_next = __ldg(n.rinfo + j_next);
            }
            uint64_t sb = ((unsigned long long)r.y << 32) | r.x;
            uint64_t se = sb + r.z;
            if (nsplit) {
                const uint32_t* sj = sp + (size_t)(j - pbase) * nsplit;
                const uint64_t beg = sb;
                if (T.tau > 0) sb = beg + __ldg(sj + T.tau - 1);
                if (T.tau < nsplit) se = beg + __ldg(sj + T.tau);
            }
            const uint32_t shift = r.w & 31u;
            int32_t* a = acc_s + ((CH == 2 && (r.w & 0x80u)) ? T.len : 0u);
            ev += se - sb;
            // edges [a4, b4) are read 4 at a time (16-byte target, 8- or 16-byte
            // weight loads); the unaligned head and tail go one edge per lane
            const uint64_t up4 = (sb + 3) & ~3ull, dn4 = se & ~3ull;
            const uint64_t a4 = up4 < se ? up4 : se;
            const uint64_t b4 = dn4 > a4 ? dn4 : a4;
            {
                uint64_t e = ~0ull;
                if (lane < a4 - sb)
                    e = sb + lane;
                else if (lane >= 4 && lane - 4 < se - b4)
                    e = b4 + (lane - 4);
                if (e != ~0ull) {
                    const uint32_t x = __ldg(n.tgt + e) - T.lo;
                    const int32_t w = weight_at<W16>(n, e, shift);
                    if (x < T.len)
                        atomicAdd(a + x, w);
                    else
                        bad = true;
                }
            }
            for (uint64_t base = a4; base < b4; base += 128 * kVec) {
                uint4 tv[kVec];
                int32_t wv[kVec][4];
#pragma unroll
                for (int u = 0; u < kVec; ++u) {
                    const uint64_t e = base + 128 * u + 4 * lane;
                    tv[u] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
                    wv[u][0] = wv[u][1] = wv[u][2] = wv[u][3] = 0;
                    if (e < b4) {
                        tv[u] = __ldg(reinterpret_cast<const uint4*>(n.tgt + e));
                        if (W16) {
                            const uint2 h = __ldg(reinterpret_cast<const uint2*>(n.w16 + e));
                            wv[u][0] = (int32_t)(int16_t)(h.x & 0xffffu) << shift;
                            wv[u][1] = (int32_t)(int16_t)(h.x >> 16) << shift;
                            wv[u][2] = (int32_t)(int16_t)(h.y & 0xffffu) << shift;
                            wv[u][3] = (int32_t)(int16_t)(h.y >> 16) << shift;
                        } else {
                            const float4 f = __ldg(reinterpret_cast<const float4*>(n.w32 + e));
                            wv[u][0] = __float2int_rz(f.x);
                            wv[u][1] = __float2int_rz(f.y);
                            wv[u][2] = __float2int_rz(f.z);
                            wv[u][3] = __float2int_rz(f.w);
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < kVec; ++u) {
                    if (base + 128 * u + 4 * lane >= b4) continue;
                    const uint32_t xs[4] = {tv[u].x - T.lo, tv[u].y - T.lo, tv[u].z - T.lo, tv[u].w - T.lo};
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        if (xs[k] < T.len)
                            atomicAdd(a + xs[k], wv[u][k]);
                        else
                            bad = true;
                    }
                }
            }
            s = s_next;
            j = j_next;
            r = r_next;
        }
        __syncthreads();
        // the tile's pending input for the next update, or this part's share of it
        int4* g0;
        int4* g1 = nullptr;
        if (T.nparts == 1) {
            g0 = reinterpret_cast<int4*>(n.acc0 + T.lo);
            if (CH == 2) g1 = reinterpret_cast<int4*>(n.acc1 + T.lo);
        } else {
            int32_t* base = partial + T.part_base + (size_t)part * CH * T.len;
            g0 = reinterpret_cast<int4*>(base);
            if (CH == 2) g1 = reinterpret_cast<int4*>(base + T.len);
        }
        int4* s0 = reinterpret_cast<int4*>(acc_s);
        for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) {
            g0[i] = s0[i];
            s0[i] = make_int4(0, 0, 0, 0);
        }
        if (CH == 2) {
            int4* s1 = reinterpret_cast<int4*>(acc_s + T.len);
            for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) {
                g1[i] = s1[i];
                s1[i] = make_int4(0, 0, 0, 0);
            }
        }
        __syncthreads();
    }
    if (lane == 0 && ev) atomicAdd(&n.ctl->events, ev);
    if (bad) atomicOr(&n.ctl->err, kErrBadTarget);
}

// Adds the parts of the multi-part tiles into the global accumulators, one
// chunk of kMergeChunk neurons per block, one int4 per thread, eight parts'
// loads in flight per thread.
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
    const uint32_t i = M.off + threadIdx.x * 4;
    if (i >= M.off + M.len) return;
    const int32_t* base = partial + T.part_base;
    for (uint32_t c = 0; c < CH; ++c) {
        const int32_t* src = base + (size_t)c * T.len + i;
        const size_t stride = (size_t)CH * T.len;  // between parts
        int4 s = make_int4(0, 0, 0, 0);
        uint32_t p = 0;
        for (; p + 8 <= T.nparts; p += 8) {
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
        for (; p < T.nparts; ++p) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(src + p * stride));
            s.x += v.x;
            s.y += v.y;
            s.z += v.z;
            s.w += v.w;
        }
        *reinterpret_cast<int4*>((c ? n.acc1 : n.acc0) + T.lo + i) = s;
    }
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
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_tiled<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    return e;
}

inline void tiled_free(TiledPlan& P, const std::function<void(void*)>& release)
{
    release(P.tiles);
    release(P.items);
    release(P.split);
    release(P.partial);
    release(P.merges);
    P = TiledPlan{};
}

// Build the plan.  work[b] is the expected delivered edges of instance b per
// step (any positive scale; null: proportional to its synapses).  An
// instance is cut by target into tiles of at most max_len padded ids (the
// shared-memory limit); a tile is split by spikes into parts so that no work
// item carries more than about total / (items_per_cta * CTAs).  Needs sorted
// rows when an instance has several tiles.
inline snn_status tiled_plan(TiledPlan& P, const Net& n, const snn_params* params, const uint32_t* pbase,
                             uint32_t n_inst, int channels, uint32_t max_len, const double* work,
                             const uint64_t* inst_edges, int sms, const std::function<void*(size_t)>& alloc,
                             const std::function<void(void*)>& release, cudaStream_t s)
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
    if (tiles.empty() || smem > (size_t)optin) return SNN_E_ARG;
    if (tiled_set_smem(smem) != cudaSuccess) return SNN_E_CUDA;
    int ctas = 0;
    cudaError_t oe = channels == 2
        ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_receive_tiled<true, 2>, kTiledThreads, smem)
        : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&ctas, k_receive_tiled<true, 1>, kTiledThreads, smem);
    if (oe != cudaSuccess || ctas < 1) {
        cudaGetLastError();
        ctas = 1;
    }
    const uint32_t n_ctas = (uint32_t)(sms * ctas);
    const double items_per_cta = 1.25;  // measured: 1-1.5 best on the batched sweep
    const double target = total > 0 ? total / (items_per_cta * n_ctas) : 1.0;
    // parts, partial buffer and the merge chunks
    struct Item {
        uint32_t code;
        double w;
    };
    std::vector<Item> items;
    std::vector<MergeDev> merges;
    unsigned long long part_total = 0;
    for (uint32_t k = 0; k < tiles.size(); ++k) {
        TileDev& d = tiles[k];
        uint32_t parts = total > 0 ? (uint32_t)std::ceil(tile_work[k] / target) : 1u;
        parts = std::max<uint32_t>(1, std::min<uint32_t>({parts, kMaxParts, n_ctas}));
        d.nparts = parts;
        if (parts > 1) {
            d.part_base = part_total;
            part_total += (unsigned long long)parts * channels * d.len;
            for (uint32_t off = 0; off < d.len; off += kMergeChunk)
                merges.push_back(MergeDev{k, off, std::min(kMergeChunk, d.len - off), 0});
        }
        for (uint32_t p = 0; p < parts; ++p) items.push_back(Item{(k << 8) | p, tile_work[k] / parts});
    }
    if (tiles.size() >= (1u << 24)) return SNN_E_ARG;
    std::stable_sort(items.begin(), items.end(), [](const Item& a, const Item& b) { return a.w > b.w; });
    std::vector<uint32_t> codes(items.size());
    for (size_t i = 0; i < items.size(); ++i) codes[i] = items[i].code;

    TiledPlan Q;
    Q.n_tiles = (uint32_t)tiles.size();
    Q.n_items = (uint32_t)codes.size();
    Q.n_merges = (uint32_t)merges.size();
    Q.max_len = longest;
    Q.channels = channels;
    Q.threads = kTiledThreads;
    Q.smem = smem;
    Q.grid = std::min<uint32_t>(Q.n_items, n_ctas);
    Q.tiles = static_cast<TileDev*>(alloc(tiles.size() * sizeof(TileDev)));
    Q.items = static_cast<uint32_t*>(alloc(codes.size() * 4));
    Q.split = static_cast<uint32_t*>(alloc(std::max<unsigned long long>(split_total, 1) * 4));
    Q.partial = static_cast<int32_t*>(alloc(std::max<unsigned long long>(part_total, 4) * 4));
    Q.merges = static_cast<MergeDev*>(alloc(std::max<size_t>(merges.size(), 1) * sizeof(MergeDev)));
    uint32_t* dbounds = static_cast<uint32_t*>(alloc(65536 * 4));
    snn_status st = (Q.tiles && Q.items && Q.split && Q.partial && Q.merges && dbounds) ? SNN_OK : SNN_E_NOMEM;
    if (st == SNN_OK &&
        (cudaMemcpyAsync(Q.tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice, s) != cudaSuccess ||
         cudaMemcpyAsync(Q.items, codes.data(), codes.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
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

inline cudaError_t enqueue_tiled_receive(const TiledPlan& P, const Net& n, bool w16, cudaStream_t s)
{
    if (P.channels == 2) {
        if (w16)
            k_receive_tiled<true, 2><<<P.grid, P.threads, P.smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len);
        else
            k_receive_tiled<false, 2><<<P.grid, P.threads, P.smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len);
        if (P.n_merges) k_merge_parts<2><<<P.n_merges, kMergeChunk / 4, 0, s>>>(n, P.tiles, P.merges, P.partial);
    } else {
        if (w16)
            k_receive_tiled<true, 1><<<P.grid, P.threads, P.smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len);
        else
            k_receive_tiled<false, 1><<<P.grid, P.threads, P.smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len);
        if (P.n_merges) k_merge_parts<1><<<P.n_merges, kMergeChunk / 4, 0, s>>>(n, P.tiles, P.merges, P.partial);
    }
    return cudaGetLastError();
}

}  // namespace snn
