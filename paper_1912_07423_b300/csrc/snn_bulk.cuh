// snn_bulk.cuh -- Receive Spikes with the rows staged by bulk asynchronous
// copies (the TMA engine) into shared memory.
//
// Same work items and accumulators as the tiled receive (snn_tiled.cuh), but
// the edges do not travel through registers: warp 0 of the CTA is a
// producer that splits the item's row segments into chunks of at most
// kBulkChunk edges and issues, per chunk, two cp.async.bulk copies (targets,
// weights) into a ring of kBulkSlots shared-memory slots, each completing the
// slot's "full" mbarrier.  Consumer warp c owns slot c: it takes the slot's
// chunks in order, reads the edges from shared memory, adds them into the
// accumulators with shared-memory atomics and releases the slot through its
// "empty" mbarrier.  Because a slot has one consumer that takes its uses in
// order (and one producer that refills it only after the release), no wait
// ever targets a phase more than one ahead -- the parity of an mbarrier
// phase cannot alias.  An item ends with one marker chunk per slot.  The
// producer keeps up to kBulkSlots chunks in flight.
//
// Copies start at 16-byte boundaries: a chunk [a, b) is copied as
// [a rounded down, b rounded up] to multiples of 4 targets / 8 int16 (or 4
// binary32) weights, and the consumer skips the extra edges.  The edge arrays
// carry 16 elements of padding so the rounded-up end stays inside them.
//
// Every wait on an mbarrier is bounded; when a bound runs out the kernel sets
// kErrTimeout, stops producing, waits (bounded) for the copies it issued, and
// returns.
#pragma once
#include <cuda_runtime.h>

#include "snn_device.cuh"
#include "snn_tiled.cuh"

namespace snn {

constexpr uint32_t kBulkChunk = 1024;  // edges per chunk
constexpr uint32_t kBulkSlots = 16;    // = consumer warps
constexpr int kBulkThreads = 32 * (kBulkSlots + 1);
constexpr uint32_t kBulkTgtBytes = (kBulkChunk + 8) * 4;
__host__ __device__ constexpr uint32_t bulk_slot_bytes(bool w16)
{
    return kBulkTgtBytes + (kBulkChunk + 16) * (w16 ? 2u : 4u);
}
constexpr uint32_t kBulkMark = 0xffffffffu;  // chunk count of an end-of-item marker
constexpr uint32_t kBulkSpin = 1u << 20;     // default bound of a producer / consumer wait (polls of try_wait)
constexpr uint32_t kBulkDrainSpin = 1u << 26; // bound of the wait for the copies in flight before exit

struct BulkMeta {
    uint32_t toff, woff, count, info;  // info: shift | channel << 8 (real); chunk total (marker)
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// true when the phase of the given parity has completed; false after `spin` polls
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t spin)
{
    const uint32_t a = smem_u32(bar);
    for (uint32_t i = 0; i < spin; ++i) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_copy(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <bool W16, int CH>
__global__ void __launch_bounds__(kBulkThreads, 1) k_receive_bulk(Net n, const TileDev* __restrict__ tiles,
                                                                  const uint32_t* __restrict__ items,
                                                                  const uint32_t* __restrict__ split,
                                                                  int32_t* __restrict__ partial, uint32_t n_items,
                                                                  uint32_t max_len, uint32_t spin)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    int32_t* acc_s = reinterpret_cast<int32_t*>(smem_raw);
    constexpr uint32_t kSlot = bulk_slot_bytes(W16);
    unsigned char* ring = smem_raw + (size_t)CH * max_len * 4;
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + kBulkSlots * kSlot);
    uint64_t* empty = full + kBulkSlots;
    BulkMeta* meta = reinterpret_cast<BulkMeta*>(empty + kBulkSlots);
    __shared__ uint32_t s_item;
    __shared__ int s_fail;

    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    constexpr uint32_t ncons = kBulkSlots;
    if (threadIdx.x == 0) {
        for (uint32_t k = 0; k < kBulkSlots; ++k) {
            mbar_init(full + k, 1);
            mbar_init(empty + k, 1);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        s_fail = 0;
    }
    __syncthreads();

    const unsigned long long t = n.ctl->t + n.k;
    unsigned int* ctr = n.tile_ctr + (t & 1ull);
    const bool deliver = t + 1 >= n.d;
    const unsigned long long ts = deliver ? t + 1 - n.d : 0ull;
    const unsigned char* gw = W16 ? reinterpret_cast<const unsigned char*>(n.w16)
                                  : reinterpret_cast<const unsigned char*>(n.w32);
    unsigned long long ev = 0;   // producer lane 0
    bool bad = false;
    uint32_t qbase = 0;          // chunk sequence number of the item's first chunk (same in every thread)
    uint32_t issued = 0;         // producer: chunks issued so far (sequence numbers < issued)

    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(ctr, 1u);
        __syncthreads();
        const uint32_t item = s_item;
        if (item >= n_items || s_fail) break;
        const uint32_t code = __ldg(items + item);
        const TileDev T = tiles[code >> 8];
        const uint32_t part = code & 0xffu;
        const uint32_t cnt = deliver ? n.icount[(size_t)(ts & (n.cr - 1)) * n.n_inst + T.inst] : 0u;
        if (cnt == 0) {  // nothing arrives: the update already cleared these accumulators
            __syncthreads();
            continue;
        }
        for (uint32_t i = threadIdx.x; i < CH * T.len; i += blockDim.x) acc_s[i] = 0;
        __syncthreads();
        const uint32_t pbase = __ldg(&n.inst[T.inst].pbase);
        const uint32_t* q = n.q + (size_t)(ts % n.D) * n.Np + pbase;
        const uint32_t nsplit = T.ntiles - 1;
        const uint32_t* sp = split + T.split;
        const uint32_t s_beg = (uint32_t)((unsigned long long)cnt * part / T.nparts);
        const uint32_t s_end = (uint32_t)((unsigned long long)cnt * (part + 1) / T.nparts);

        if (warp == 0) {
            // ---------------- producer ----------------
            uint32_t K = 0;  // real chunks of this item
            bool ok = true;
            for (uint32_t s0 = s_beg; s0 < s_end && ok; s0 += 32) {
                // 32 spikes' segments in parallel
                const uint32_t s = s0 + lane;
                uint64_t sb = 0, se = 0;
                uint32_t info = 0;
                if (s < s_end) {
                    const uint32_t j = q[s];
                    const uint4 r = __ldg(n.rinfo + j);
                    sb = ((unsigned long long)r.y << 32) | r.x;
                    se = sb + r.z;
                    if (nsplit) {
                        const uint32_t* sj = sp + (size_t)(j - pbase) * nsplit;
                        const uint64_t beg = sb;
                        if (T.tau > 0) sb = beg + __ldg(sj + T.tau - 1);
                        if (T.tau < nsplit) se = beg + __ldg(sj + T.tau);
                    }
                    info = (r.w & 31u) | ((CH == 2 && (r.w & 0x80u)) ? 0x100u : 0u);
                }
                const uint32_t nlanes = min(32u, s_end - s0);
                for (uint32_t l = 0; l < nlanes; ++l) {
                    const uint64_t a0 = __shfl_sync(0xffffffffu, sb, l);
                    const uint64_t b0 = __shfl_sync(0xffffffffu, se, l);
                    const uint32_t inf = __shfl_sync(0xffffffffu, info, l);
                    if (lane == 0) ev += b0 - a0;
                    for (uint64_t a = a0; a < b0 && ok; a += kBulkChunk) {
                        const uint64_t b = a + kBulkChunk < b0 ? a + kBulkChunk : b0;
                        if (lane == 0) {
                            const uint32_t qn = issued;
                            const uint32_t slot = qn % kBulkSlots, use = qn / kBulkSlots;
                            if (use > 0 && !mbar_wait(empty + slot, (use - 1) & 1u, spin)) ok = false;
                            if (ok) {
                                const uint64_t ta = a & ~3ull, tb = (b + 3) & ~3ull;
                                const uint64_t wa = W16 ? (a & ~7ull) : ta;
                                const uint64_t wb = W16 ? ((b + 7) & ~7ull) : tb;
                                const uint32_t tbytes = (uint32_t)(tb - ta) * 4u;
                                const uint32_t wbytes = (uint32_t)(wb - wa) * (W16 ? 2u : 4u);
                                meta[slot] = BulkMeta{(uint32_t)(a - ta), (uint32_t)(a - wa), (uint32_t)(b - a), inf};
                                unsigned char* dst = ring + (size_t)slot * kSlot;
                                mbar_arrive_tx(full + slot, tbytes + wbytes);
                                bulk_copy(dst, n.tgt + ta, tbytes, full + slot);
                                bulk_copy(dst + kBulkTgtBytes, gw + wa * (W16 ? 2u : 4u), wbytes, full + slot);
                                issued = qn + 1;
                                ++K;
                            }
                        }
                        ok = __shfl_sync(0xffffffffu, ok, 0);
                    }
                }
            }
            // one end marker per slot (= per consumer warp), carrying the chunk total
            for (uint32_t m = 0; m < ncons && ok; ++m) {
                if (lane == 0) {
                    const uint32_t qn = issued;
                    const uint32_t slot = qn % kBulkSlots, use = qn / kBulkSlots;
                    if (use > 0 && !mbar_wait(empty + slot, (use - 1) & 1u, spin)) ok = false;
                    if (ok) {
                        meta[slot] = BulkMeta{0, 0, kBulkMark, K};
                        mbar_arrive(full + slot);
                        issued = qn + 1;
                    }
                }
                ok = __shfl_sync(0xffffffffu, ok, 0);
            }
            if (!ok && lane == 0) {
                s_fail = 1;
                atomicOr(&n.ctl->err, kErrTimeout);
            }
            qbase = __shfl_sync(0xffffffffu, issued, 0);  // the next item starts after the markers
        } else {
            // ---------------- consumers ----------------
            // warp c (c = warp - 1) owns slot c: chunks qn = c (mod kBulkSlots)
            const uint32_t c = warp - 1;
            uint32_t qn = qbase + (c + kBulkSlots - qbase % kBulkSlots) % kBulkSlots;
            for (;;) {
                const uint32_t slot = c, use = qn / kBulkSlots;
                // every lane waits, so every lane acquires the chunk's data
                bool ok = mbar_wait(full + slot, use & 1u, spin);
                ok = __shfl_sync(0xffffffffu, ok, 0);
                if (!ok) {
                    if (lane == 0) {
                        s_fail = 1;
                        atomicOr(&n.ctl->err, kErrTimeout);
                    }
                    break;
                }
                const BulkMeta M = meta[slot];
                if (M.count == kBulkMark) {
                    __syncwarp();
                    if (lane == 0) mbar_arrive(empty + slot);
                    qbase = qbase + M.info + kBulkSlots;
                    break;
                }
                const uint32_t* st = reinterpret_cast<const uint32_t*>(ring + (size_t)slot * kSlot) + M.toff;
                const unsigned char* sw = ring + (size_t)slot * kSlot + kBulkTgtBytes;
                const uint32_t shift = M.info & 31u;
                int32_t* a = acc_s + ((CH == 2 && (M.info & 0x100u)) ? T.len : 0u);
                for (uint32_t k = lane; k < M.count; k += 32) {
                    const uint32_t x = st[k] - T.lo;
                    const int32_t w = W16 ? ((int32_t)reinterpret_cast<const int16_t*>(sw)[M.woff + k] << shift)
                                          : __float2int_rz(reinterpret_cast<const float*>(sw)[M.woff + k]);
                    if (x < T.len)
                        atomicAdd(a + x, w);
                    else
                        bad = true;
                }
                __syncwarp();
                if (lane == 0) {
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    mbar_arrive(empty + slot);
                }
                qn += kBulkSlots;
            }
        }
        __syncthreads();
        if (s_fail) break;
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
        const int4* s0 = reinterpret_cast<const int4*>(acc_s);
        for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) g0[i] = s0[i];
        if (CH == 2) {
            const int4* s1 = reinterpret_cast<const int4*>(acc_s + T.len);
            for (uint32_t i = threadIdx.x; i < T.len / 4; i += blockDim.x) g1[i] = s1[i];
        }
        __syncthreads();
    }
    // leave no copy in flight: wait for the last use of every slot.  Issued
    // copies always complete, so this wait ends unless the memory system has
    // failed; its bound (kBulkDrainSpin, far above any copy's latency) only
    // keeps the kernel from spinning forever then, and is reported as a timeout
    if (threadIdx.x == 0 && issued > 0) {
        const uint32_t first = issued > kBulkSlots ? issued - kBulkSlots : 0;
        for (uint32_t qn = first; qn < issued; ++qn)
            if (!mbar_wait(full + qn % kBulkSlots, (qn / kBulkSlots) & 1u, kBulkDrainSpin))
                atomicOr(&n.ctl->err, kErrTimeout);
    }
    if (threadIdx.x == 0 && ev) atomicAdd(&n.ctl->events, ev);
    if (bad) atomicOr(&n.ctl->err, kErrBadTarget);
}

inline size_t bulk_smem(uint32_t max_len, int channels, bool w16)
{
    return (size_t)channels * max_len * 4 + (size_t)kBulkSlots * bulk_slot_bytes(w16) + 2 * kBulkSlots * 8 +
           kBulkSlots * sizeof(BulkMeta);
}

inline cudaError_t bulk_set_smem(size_t smem)
{
    cudaError_t e = cudaSuccess;
    const int s = (int)smem;
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_bulk<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_bulk<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_bulk<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_receive_bulk<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, s);
    return e;
}

inline cudaError_t enqueue_bulk_receive(const TiledPlan& P, const Net& n, bool w16, cudaStream_t s, uint32_t spin,
                                        cudaEvent_t mid = nullptr /* recorded between the receive and the merge */)
{
    const size_t smem = bulk_smem(P.max_len, P.channels, w16);
    if (P.channels == 2) {
        if (w16)
            k_receive_bulk<true, 2><<<P.grid, kBulkThreads, smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len, spin);
        else
            k_receive_bulk<false, 2><<<P.grid, kBulkThreads, smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len, spin);
        if (mid) cudaEventRecord(mid, s);
        if (P.n_merges) k_merge_parts<2><<<P.n_merges, kMergeChunk / 4, 0, s>>>(n, P.tiles, P.merges, P.partial);
    } else {
        if (w16)
            k_receive_bulk<true, 1><<<P.grid, kBulkThreads, smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len, spin);
        else
            k_receive_bulk<false, 1><<<P.grid, kBulkThreads, smem, s>>>(n, P.tiles, P.items, P.split, P.partial, P.n_items, P.max_len, spin);
        if (mid) cudaEventRecord(mid, s);
        if (P.n_merges) k_merge_parts<1><<<P.n_merges, kMergeChunk / 4, 0, s>>>(n, P.tiles, P.merges, P.partial);
    }
    return cudaGetLastError();
}

}  // namespace snn
