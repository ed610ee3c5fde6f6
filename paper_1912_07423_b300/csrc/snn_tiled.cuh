// snn_tiled.cuh -- Receive Spikes with the accumulators in shared memory.
//
// The paper delivers a spike with one CUDA block walking the spiker's
// adjacency row and updating the recipients with atomics (Section III-A-2).
// On a B300 the random 32-bit red.global.add that such a walk issues runs at
// about 2e11 per second into L2, a fifth of what HBM can stream in edges, so
// this form divides the work by TARGET instead: every network instance is cut
// into tiles of consecutive neuron ids small enough for one CTA's shared
// memory.  The CTA of a tile walks every spike of its instance, reads only the
// segment of the spiker's (sorted) row that falls inside the tile, adds the
// weights with shared-memory atomics, and finally stores the whole tile to
// the global accumulators with coalesced writes.  Each edge is read once per
// step; no global atomics are issued.  Segment bounds of rows that span
// several tiles come from a split table built once with the graph.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "../../include/snn.h"
#include "snn_device.cuh"

namespace snn {

struct TileDev {
    uint32_t inst;            // instance
    uint32_t lo, len;         // padded id range [lo, lo + len); len is a multiple of 256
    uint32_t tau, ntiles;     // tile index inside the instance, tiles of the instance
    uint32_t pad;
    unsigned long long split; // base of the instance's split table: (ntiles-1) x n_b uint32
};

struct TiledPlan {
    TileDev* tiles = nullptr;
    uint32_t* split = nullptr;
    uint32_t n_tiles = 0;
    uint32_t max_len = 0;
    int channels = 1;
    int threads = 512;
    size_t smem = 0;
};

constexpr int kTiledThreads = 512;

template <bool W16, int CH>
__global__ void __launch_bounds__(kTiledThreads) k_receive_tiled(Net n, const TileDev* __restrict__ tiles,
                                                                 const uint32_t* __restrict__ split)
{
    extern __shared__ int32_t acc_s[];  // CH * len
    const TileDev T = tiles[blockIdx.x];
    for (uint32_t i = threadIdx.x; i < CH * T.len; i += blockDim.x) acc_s[i] = 0;
    __syncthreads();
    const unsigned long long t = n.ctl->t;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    unsigned long long ev = 0;
    bool bad = false;  // a target outside the tile: the split table does not match the rows
    if (t + 1 >= n.d) {
        const unsigned long long ts = t + 1 - n.d;
        const uint32_t cnt = n.icount[(size_t)(ts & (n.cr - 1)) * n.n_inst + T.inst];
        const InstDev* I = n.inst + T.inst;
        const uint32_t pbase = __ldg(&I->pbase), nb = __ldg(&I->n);
        const uint32_t* q = n.q + (size_t)(ts % n.D) * n.Np + pbase;
        const uint32_t* s_lo = T.tau > 0 ? split + T.split + (size_t)(T.tau - 1) * nb : nullptr;
        const uint32_t* s_hi = T.tau + 1 < T.ntiles ? split + T.split + (size_t)T.tau * nb : nullptr;
        for (uint32_t s = warp; s < cnt; s += nwarps) {
            const uint32_t j = q[s];
            const uint64_t beg = __ldg(n.roff + j), end = __ldg(n.roff + j + 1);
            uint64_t sb = beg, se = end;
            if (s_lo) sb = beg + __ldg(s_lo + (j - pbase));
            if (s_hi) se = beg + __ldg(s_hi + (j - pbase));
            const uint32_t meta = __ldg(n.meta + j);
            const uint32_t shift = meta & 31u;
            int32_t* a = acc_s + ((CH == 2 && (meta & 0x80u)) ? T.len : 0u) - T.lo;
            ev += se - sb;
            uint64_t e = sb + lane;
            for (; e + 96 < se; e += 128) {
                uint32_t tg[4];
                int32_t wv[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    tg[u] = __ldg(n.tgt + e + 32 * u);
                    wv[u] = W16 ? ((int32_t)__ldg(n.w16 + e + 32 * u) << shift)
                                : __float2int_rz(__ldg(n.w32 + e + 32 * u));
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (tg[u] - T.lo < T.len)
                        atomicAdd(a + tg[u], wv[u]);
                    else
                        bad = true;
                }
            }
            for (; e < se; e += 32) {
                const uint32_t tg = __ldg(n.tgt + e);
                const int32_t wv = W16 ? ((int32_t)__ldg(n.w16 + e) << shift) : __float2int_rz(__ldg(n.w32 + e));
                if (tg - T.lo < T.len)
                    atomicAdd(a + tg, wv);
                else
                    bad = true;
            }
        }
    }
    __syncthreads();
    // the tile's pending input for the next update (whole tile, every step)
    int4* g0 = reinterpret_cast<int4*>(n.acc0 + T.lo);
    const int4* s0 = reinterpret_cast<const int4*>(acc_s);
    for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) g0[i] = s0[i];
    if (CH == 2) {
        int4* g1 = reinterpret_cast<int4*>(n.acc1 + T.lo);
        const int4* s1 = reinterpret_cast<const int4*>(acc_s + T.len);
        for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) g1[i] = s1[i];
    }
    // every lane of a warp counted the same segments: lane 0 reports them
    if (lane == 0 && ev) atomicAdd(&n.ctl->events, ev);
    if (bad) atomicOr(&n.ctl->err, kErrBadTarget);
}

// Split table: for row j of a multi-tile instance and inner boundary tau,
// the offset inside the row of the first target >= the boundary's padded id.
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
            split[(size_t)(tau - 1) * nb + l] = (uint32_t)(lo - beg);
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

// Cut every instance into tiles of at most max_len padded ids (multiples of
// 256) and build the split tables of the instances with several tiles.
// tiles_per_inst, if given, asks for at least that many tiles per instance
// (load balancing by expected work).  Needs sorted rows.
inline snn_status tiled_plan(TiledPlan& P, const Net& n, const snn_params* params, const uint32_t* pbase,
                             uint32_t n_inst, int channels, uint32_t max_len, const uint32_t* tiles_per_inst,
                             const std::function<void*(size_t)>& alloc, const std::function<void(void*)>& release,
                             cudaStream_t s)
{
    max_len = std::max<uint32_t>(256, max_len / 256 * 256);
    std::vector<TileDev> tiles;
    std::vector<std::vector<uint32_t>> bounds(n_inst);
    unsigned long long split_total = 0;
    for (uint32_t b = 0; b < n_inst; ++b) {
        const uint32_t npad = pbase[b + 1] - pbase[b];
        if (npad == 0) continue;
        const uint32_t m = npad / 256;
        uint32_t T = (npad + max_len - 1) / max_len;
        if (tiles_per_inst) T = std::max(T, tiles_per_inst[b]);
        T = std::min(T, m);
        auto& B = bounds[b];
        B.resize(T + 1);
        for (uint32_t tau = 0; tau <= T; ++tau) B[tau] = pbase[b] + 256u * (uint32_t)((unsigned long long)tau * m / T);
        for (uint32_t tau = 0; tau < T; ++tau) {
            TileDev d{};
            d.inst = b;
            d.lo = B[tau];
            d.len = B[tau + 1] - B[tau];
            d.tau = tau;
            d.ntiles = T;
            d.split = split_total;
            tiles.push_back(d);
        }
        if (T > 1) split_total += (unsigned long long)(T - 1) * params[b].n;
    }
    uint32_t longest = 0;
    for (const TileDev& d : tiles) longest = std::max(longest, d.len);
    P.n_tiles = (uint32_t)tiles.size();
    P.max_len = longest;
    P.channels = channels;
    P.threads = kTiledThreads;
    P.smem = (size_t)longest * channels * 4;
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (P.smem > (size_t)optin || P.n_tiles == 0) return SNN_E_ARG;
    if (tiled_set_smem(P.smem) != cudaSuccess) return SNN_E_CUDA;
    P.tiles = static_cast<TileDev*>(alloc(tiles.size() * sizeof(TileDev)));
    P.split = static_cast<uint32_t*>(alloc(std::max<unsigned long long>(split_total, 1) * 4));
    if (!P.tiles || !P.split) return SNN_E_NOMEM;
    struct Tmp {
        uint32_t* p;
        const std::function<void(void*)>& f;
        ~Tmp() { f(p); }
    } dbounds{static_cast<uint32_t*>(alloc(65536 * 4)), release};
    if (!dbounds.p) return SNN_E_NOMEM;
    if (cudaMemcpyAsync(P.tiles, tiles.data(), tiles.size() * sizeof(TileDev), cudaMemcpyHostToDevice, s) != cudaSuccess)
        return SNN_E_CUDA;
    for (uint32_t b = 0; b < n_inst; ++b) {
        const auto& B = bounds[b];
        if (B.size() <= 2) continue;
        const uint32_t T = (uint32_t)B.size() - 1;
        if (T + 1 > 65536) return SNN_E_ARG;
        unsigned long long base = 0;
        for (const TileDev& d : tiles)
            if (d.inst == b) {
                base = d.split;
                break;
            }
        if (cudaMemcpyAsync(dbounds.p, B.data(), B.size() * 4, cudaMemcpyHostToDevice, s) != cudaSuccess) return SNN_E_CUDA;
        k_split_rows<<<1184, 256, 0, s>>>(n.roff, n.tgt, pbase[b], params[b].n, dbounds.p, T, P.split + base);
        if (cudaGetLastError() != cudaSuccess) return SNN_E_CUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return SNN_E_CUDA;
    }
    return SNN_OK;
}

inline cudaError_t enqueue_tiled_receive(const TiledPlan& P, const Net& n, bool w16, cudaStream_t s)
{
    if (P.channels == 2) {
        if (w16)
            k_receive_tiled<true, 2><<<P.n_tiles, P.threads, P.smem, s>>>(n, P.tiles, P.split);
        else
            k_receive_tiled<false, 2><<<P.n_tiles, P.threads, P.smem, s>>>(n, P.tiles, P.split);
    } else {
        if (w16)
            k_receive_tiled<true, 1><<<P.n_tiles, P.threads, P.smem, s>>>(n, P.tiles, P.split);
        else
            k_receive_tiled<false, 1><<<P.n_tiles, P.threads, P.smem, s>>>(n, P.tiles, P.split);
    }
    return cudaGetLastError();
}

}  // namespace snn

namespace snn {
inline void tiled_free(TiledPlan& P, const std::function<void(void*)>& release)
{
    release(P.tiles);
    release(P.split);
    P = TiledPlan{};
}
}  // namespace snn
