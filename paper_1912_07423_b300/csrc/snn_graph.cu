// snn_graph.cu -- adjacency construction on the GPU (Section III-A-2, Fig. 2).
//
// A job (n, a, b, o) asks for n sorted, unique, uniformly distributed random
// integers from [a, b), written at out[o .. o + n).  The running sums of
// exponentially distributed spacings are, once normalised by their total,
// the order statistics of uniform draws; scaled to b - a - n and rounded,
// with 0 .. n-1 added to keep them distinct, they are the job's values.
//
// One warp per job.  Uniforms u_k, k = 0..n (n + 1 spacings, the figure's
// two sentinels being the zero start and the normalising total), come from
// Philox4x64-10 with key (seed, job) and counter (k >> 3, 0, 2, 0), word
// k & 7: u_k = ((word >> 8) + 1) 2^-24 in (0, 1].  The spacing -ln u_k is
// computed in binary32 by this file's own logarithm (range reduction to
// m in [1, 2) from the bits, ln m = 2 s (1 + s^2/3 + ... + s^12/13) by
// Horner's rule, s = (m - 1) / (m + 1)) and held as an integer q_k =
// round(-ln u_k 2^22), so that running sums are exact in any order (and 32
// of them fit 32 bits).  Pass 1 draws the spacings (a lane per Philox block
// of 8), sums them and parks q_0 .. q_{n-1} in the job's own output slots
// (through shared memory, so the stores are coalesced); pass 2 reads them
// back 256 at a time, sums each lane's 8, scans the lanes' sums across the
// warp and overwrites slot k with a + round(c_{k+1} f) + k, c the exclusive
// running sum and f = (b - a - n) / total (binary32, at most b - a - n).  Every operation is rounded as
// written (-fmad=false), so the values do not depend on the launch.  A job
// of at most 1,024 spacings (n <= 1023, the rows of the networks here) takes
// one pass instead: the lanes draw the Philox blocks in turn into shared
// memory, lane l takes spacings 32 l .. 32 l + 31 from there, the lanes'
// sums are scanned, each lane turns its 32 running sums into values, and
// the values leave through shared memory in coalesced stores -- the output
// is written once.
#include <cuda_runtime.h>


#include "../../include/snn.h"
#include "snn_device.cuh"

namespace {

constexpr unsigned kJobThreads = 256;
constexpr uint32_t kOnePass = 1024;  // most spacings (n + 1) a job takes in one pass: 32 per lane
constexpr uint32_t kMaxScale = 1u << 24;  // b - a - n: the binary32 ratio keeps every integer below it apart

// flag of an invalid job, one per device (no allocation)
static __device__ unsigned int g_job_err;

__device__ __forceinline__ float neg_ln_f32(float u)
{
    const uint32_t bits = __float_as_uint(u);
    const int32_t e = (int32_t)((bits >> 23) & 0xffu) - 127;
    const float m = __uint_as_float((bits & 0x7fffffu) | 0x3f800000u);
    const float s = __fdiv_rn(__fsub_rn(m, 1.0f), __fadd_rn(m, 1.0f));
    const float s2 = __fmul_rn(s, s);
    float p = 1.0f / 13.0f;
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f / 11.0f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f / 9.0f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f / 7.0f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f / 5.0f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f / 3.0f);
    p = __fadd_rn(__fmul_rn(p, s2), 1.0f);
    return -__fadd_rn(__fmul_rn(__int2float_rn(e), 0.693147182f), __fmul_rn(2.0f, __fmul_rn(s, p)));
}

// the 8 integer spacings of Philox block g of job j (k = 8g .. 8g + 7)
__device__ __forceinline__ void spacings8(uint64_t seed, uint32_t j, uint32_t g, uint32_t q[8])
{
    uint32_t w[8];
    snn::philox_words8(seed, j, g, 0, 2, w);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const float u = __fmul_rn(__uint2float_rn((w[i] >> 8) + 1u), 1.0f / 16777216.0f);
        q[i] = __float2uint_rz(__fadd_rn(__fmul_rn(neg_ln_f32(u), 4194304.0f), 0.5f));
    }
}

// a warp's 256 values in shared memory: value k (0..255) at (k / 8) 9 + k % 8,
// so that lane l's 8 consecutive values and the 32 values of one coalesced
// access both fall in (nearly) distinct banks
__device__ __forceinline__ uint32_t stage_at(uint32_t k) { return (k >> 3) * 9u + (k & 7u); }

// Jobs of at most kOnePass spacings, one pass each (see the file's header).
__global__ void __launch_bounds__(kJobThreads) k_expand_short(const snn_job* __restrict__ jobs, uint64_t n_jobs,
                                                              uint64_t seed, uint32_t* __restrict__ out,
                                                              uint64_t out_len)
{
    __shared__ uint32_t stage1[kJobThreads / 32][kOnePass + 32];  // value k at k + k / 32
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* st1 = stage1[threadIdx.x >> 5];
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t jj = warp; jj < n_jobs; jj += nwarps) {
        const snn_job J = jobs[jj];
        const uint32_t j = (uint32_t)jj;
        if (J.b < J.a || J.n > J.b - J.a || J.b - J.a - J.n > kMaxScale || J.o > out_len || J.n > out_len - J.o)
            continue;  // reported by k_expand_jobs
        const uint32_t n = J.n, M = J.b - J.a - J.n;
        if (n == 0 || n >= kOnePass) continue;
        uint32_t* dst = out + J.o;
        // draw: lane l takes Philox blocks l, l + 32, ... (spacings 8 g .. 8 g + 7)
#pragma unroll 1
        for (uint32_t g = lane; g * 8 <= n; g += 32) {
            uint32_t w8[8];
            spacings8(seed, j, g, w8);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint32_t k = 8 * g + i;
                st1[k + (k >> 5)] = w8[i];
            }
        }
        __syncwarp();
        // lane l: spacings 32 l .. 32 l + 31 (none beyond n), summed, then
        // replaced in place by their values
        unsigned long long s32 = 0;
#pragma unroll 8
        for (int i = 0; i < 32; ++i)
            if (32 * lane + i <= n) s32 += st1[33 * lane + i];
        unsigned long long incl = s32;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (uint32_t)o) incl += y;
        }
        const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
        const float f = total ? __fdiv_rn(__uint2float_rn(M), __ull2float_rn(total)) : 0.0f;
        unsigned long long c = incl - s32;
#pragma unroll 1
        for (int i = 0; i < 32; ++i) {
            const uint32_t k = 32 * lane + i;
            if (k >= n) break;
            c += st1[33 * lane + i];  // c_{k+1}
            uint32_t r = __float2uint_rz(__fadd_rn(__fmul_rn(__ull2float_rn(c), f), 0.5f));
            r = r > M ? M : r;
            st1[33 * lane + i] = J.a + r + k;
        }
        __syncwarp();
#pragma unroll
        for (int i = 0; i < 32; ++i) {
            const uint32_t k = 32 * i + lane;
            if (k < n) dst[k] = st1[33 * i + lane];
        }
        __syncwarp();
    }
}

__global__ void __launch_bounds__(kJobThreads) k_expand_jobs(const snn_job* __restrict__ jobs, uint64_t n_jobs,
                                                             uint64_t seed, uint32_t* __restrict__ out,
                                                             uint64_t out_len)
{
    __shared__ uint32_t stage[kJobThreads / 32][32 * 9];
    const uint32_t lane = threadIdx.x & 31u;
    uint32_t* st = stage[threadIdx.x >> 5];
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t jj = warp; jj < n_jobs; jj += nwarps) {
        const snn_job J = jobs[jj];
        const uint32_t j = (uint32_t)jj;
        if (J.b < J.a || J.n > J.b - J.a || J.b - J.a - J.n > kMaxScale || J.o > out_len || J.n > out_len - J.o) {
            if (lane == 0) atomicOr(&g_job_err, 1u);
            continue;
        }
        const uint32_t n = J.n, M = J.b - J.a - J.n;
        if (n == 0) continue;
        uint32_t* dst = out + J.o;
        if (n < kOnePass) continue;  // k_expand_short's

        // pass 1: the total of the n + 1 spacings; q_0 .. q_{n-1} parked in
        // the output (lane l draws block l of every 256 spacings)
        unsigned long long part = 0;
        for (uint64_t base = 0; base <= n; base += 256) {
            const uint32_t g = (uint32_t)(base >> 3) + lane;
            uint32_t q[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            if ((uint64_t)g * 8 <= n) spacings8(seed, j, g, q);
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                if ((uint64_t)g * 8 + i > n) q[i] = 0;
                part += q[i];
                st[lane * 9 + i] = q[i];
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t k = base + 32 * i + lane;
                if (k < n) dst[k] = st[stage_at(32 * i + lane)];
            }
            __syncwarp();
        }
#pragma unroll
        for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const float f = part ? __fdiv_rn(__uint2float_rn(M), __ull2float_rn(part)) : 0.0f;
        // pass 2, 256 at a time: lane l takes 8 consecutive spacings, sums
        // them, and the lanes' sums are scanned across the warp; slot k gets
        // a + round(c_{k+1} f) + k, c_{k+1} the running sum through q_k
        unsigned long long carry = 0;
        for (uint64_t base = 0; base < n; base += 256) {
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t k = base + 32 * i + lane;
                st[stage_at(32 * i + lane)] = k < n ? dst[k] : 0u;
            }
            __syncwarp();
            uint32_t v[8];
            unsigned long long s8 = 0;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                v[i] = st[lane * 9 + i];
                s8 += v[i];
            }
            unsigned long long incl = s8;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= (uint32_t)o) incl += y;
            }
            unsigned long long c = carry + incl - s8;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                c += v[i];  // c_{k+1}, k = base + 8 lane + i
                uint32_t r = __float2uint_rz(__fadd_rn(__fmul_rn(__ull2float_rn(c), f), 0.5f));
                r = r > M ? M : r;
                st[lane * 9 + i] = J.a + r + (uint32_t)(base + 8 * lane + i);
            }
            __syncwarp();
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const uint64_t k = base + 32 * i + lane;
                if (k < n) dst[k] = st[stage_at(32 * i + lane)];
            }
            __syncwarp();
            carry += __shfl_sync(0xffffffffu, incl, 31);
        }
    }
}

}  // namespace

extern "C" snn_status snn_expand_jobs(const snn_job* jobs, uint64_t n_jobs, uint64_t seed, uint32_t* out,
                                      uint64_t out_len, void* stream)
{
    if (n_jobs == 0) return SNN_OK;
    if (!jobs || (!out && out_len) || n_jobs > 0xffffffffull) return SNN_E_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned int* err = nullptr;
    if (cudaGetSymbolAddress((void**)&err, g_job_err) != cudaSuccess) {
        cudaGetLastError();
        return SNN_E_CUDA;
    }
    if (cudaMemsetAsync(err, 0, sizeof(unsigned int), s) != cudaSuccess) return SNN_E_CUDA;
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const uint64_t warps_needed = n_jobs;
    const uint64_t blocks = (warps_needed * 32 + kJobThreads - 1) / kJobThreads;
    const uint32_t grid = (uint32_t)(blocks < (uint64_t)sms * 16 ? blocks : (uint64_t)sms * 16);
    k_expand_short<<<grid, kJobThreads, 0, s>>>(jobs, n_jobs, seed, out, out_len);
    k_expand_jobs<<<grid, kJobThreads, 0, s>>>(jobs, n_jobs, seed, out, out_len);
    if (cudaGetLastError() != cudaSuccess) return SNN_E_CUDA;
    unsigned int h = 0;
    if (cudaMemcpyAsync(&h, err, sizeof h, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return SNN_E_CUDA;
    return h ? SNN_E_ARG : SNN_OK;
}
