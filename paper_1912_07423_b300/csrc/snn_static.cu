// snn_static.cu -- population rate and ISI CV without any device allocation.
//
// snn_stats reduces the per-neuron spike statistics into a few doubles of
// scratch that it takes from the context's allocator on every call.  Some
// callers cannot allocate device memory at the moment they want these
// numbers: an application that hands the whole GPU to its own fixed memory
// arena at start-up (a stray cudaMalloc there fails or fragments the arena),
// or a latency-critical loop where cudaMalloc/cudaFree may synchronise the
// device and stall every other stream.  snn_rate_cv_static serves them: its
// scratch is the file-scope array below, which every GPU that loads this
// library holds until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "../../include/snn.h"

namespace {

constexpr unsigned kNeuronsPerBlock = 2048;  // one block reduces this many neurons
constexpr unsigned kMaxBlocks = 8192;        // => at most 16,777,216 neurons per call
constexpr unsigned kThreads = 256;

// Per-block partial sums (spikes, sum of CVs, neurons with >= 3 spikes),
// then the 3 final values in the last slots: 8192*3 + 3 doubles = 192 KB.
static __device__ __align__(256) double g_rate_cv_scratch[3 * kMaxBlocks + 3];

// Block b reduces neurons [b*2048, min(n, (b+1)*2048)) into partial[3b..3b+2].
// Every slot a call reads is written earlier in the same call, so the array
// needs no clearing between calls.
__global__ void __launch_bounds__(kThreads) k_rate_cv_partial(const uint32_t* cnt, const unsigned long long* sum,
                                                               const unsigned long long* sq, uint32_t n,
                                                               double* partial)
{
    __shared__ double red[3][kThreads];
    double s_spk = 0.0, s_cv = 0.0, s_n = 0.0;
    const uint32_t lo = blockIdx.x * kNeuronsPerBlock;
    const uint32_t hi = min(n, lo + kNeuronsPerBlock);
    for (uint32_t i = lo + threadIdx.x; i < hi; i += kThreads) {
        const uint32_t c = cnt[i];
        s_spk += (double)c;
        if (c >= 3) {
            const double m = (double)sum[i] / (double)(c - 1);
            const double var = (double)sq[i] / (double)(c - 1) - m * m;
            s_cv += sqrt(var > 0.0 ? var : 0.0) / m;
            s_n += 1.0;
        }
    }
    red[0][threadIdx.x] = s_spk;
    red[1][threadIdx.x] = s_cv;
    red[2][threadIdx.x] = s_n;
    __syncthreads();
    for (unsigned o = kThreads / 2; o; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) partial[3 * blockIdx.x + threadIdx.x] = red[threadIdx.x][0];
}

// One block adds the partials in a fixed order into the last 3 slots.
__global__ void __launch_bounds__(kThreads) k_rate_cv_final(double* scratch, uint32_t nblocks)
{
    __shared__ double red[3][kThreads];
    double a[3] = {0.0, 0.0, 0.0};
    for (uint32_t b = threadIdx.x; b < nblocks; b += kThreads)
        for (int k = 0; k < 3; ++k) a[k] += scratch[3 * b + k];
    for (int k = 0; k < 3; ++k) red[k][threadIdx.x] = a[k];
    __syncthreads();
    for (unsigned o = kThreads / 2; o; o >>= 1) {
        if (threadIdx.x < o)
            for (int k = 0; k < 3; ++k) red[k][threadIdx.x] += red[k][threadIdx.x + o];
        __syncthreads();
    }
    if (threadIdx.x < 3) scratch[3 * kMaxBlocks + threadIdx.x] = red[threadIdx.x][0];
}

// Device address of the scratch array, looked up once per device and CUDA
// context: a cudaDeviceReset destroys the device's primary context and the
// module with it, so an address cached for the old context would point into
// freed memory.  The context is told apart by its process-unique id
// (cuCtxGetId), reached through the runtime's driver entry points so that the
// library does not link the driver library itself.
constexpr int kMaxDevices = 64;
struct ScratchSlot {
    unsigned long long ctx_id;
    double* addr;
};
std::mutex g_mu;
ScratchSlot g_slot[kMaxDevices] = {};

using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id)
{
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    if (!get_current || !get_id) {
        void* f0 = nullptr;
        void* f1 = nullptr;
        cudaDriverEntryPointQueryResult q0{}, q1{};
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f0, 12000, cudaEnableDefault, &q0);
        if (e == cudaSuccess) e = cudaGetDriverEntryPointByVersion("cuCtxGetId", &f1, 12000, cudaEnableDefault, &q1);
        if (e != cudaSuccess) return e;
        if (q0 != cudaDriverEntryPointSuccess || q1 != cudaDriverEntryPointSuccess || !f0 || !f1)
            return cudaErrorNotSupported;
        get_current = reinterpret_cast<CtxGetCurrentFn>(f0);
        get_id = reinterpret_cast<CtxGetIdFn>(f1);
    }
    CUcontext ctx = nullptr;
    if (get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
    return cudaSuccess;
}

cudaError_t scratch_address(double** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    // make the device's primary context current on this thread (the runtime
    // creates it here if nothing has used the device yet)
    e = cudaSetDevice(dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_mu);
    unsigned long long id = 0;
    e = current_context_id(&id);
    if (e != cudaSuccess) return e;
    ScratchSlot& slot = g_slot[dev];
    if (!slot.addr || slot.ctx_id != id) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_rate_cv_scratch);
        if (e != cudaSuccess) return e;
        slot.addr = static_cast<double*>(p);
        slot.ctx_id = id;
    }
    *out = slot.addr;
    return cudaSuccess;
}

}  // namespace

extern "C" snn_status snn_rate_cv_static(const uint32_t* count, const unsigned long long* isi_sum,
                                         const unsigned long long* isi_sq, uint32_t n, uint64_t window_steps,
                                         double dt_ms, void* stream, double* rate_hz, double* isi_cv)
{
    if (!rate_hz || !isi_cv) return SNN_E_ARG;
    if (n > kNeuronsPerBlock * kMaxBlocks) return SNN_E_ARG;  // beyond what the static scratch holds
    if (n > 0 && (!count || !isi_sum || !isi_sq)) return SNN_E_ARG;
    if (!(dt_ms > 0.0)) return SNN_E_ARG;
    *rate_hz = 0.0;
    *isi_cv = 0.0;
    if (n == 0) return SNN_OK;
    double* scratch = nullptr;
    if (scratch_address(&scratch) != cudaSuccess) {
        cudaGetLastError();
        return SNN_E_CUDA;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const uint32_t nblocks = (n + kNeuronsPerBlock - 1) / kNeuronsPerBlock;
    k_rate_cv_partial<<<nblocks, kThreads, 0, s>>>(count, isi_sum, isi_sq, n, scratch);
    k_rate_cv_final<<<1, kThreads, 0, s>>>(scratch, nblocks);
    double h[3] = {0.0, 0.0, 0.0};
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, scratch + 3 * kMaxBlocks, sizeof h, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return SNN_E_CUDA;
    }
    const double window_s = (double)window_steps * dt_ms * 1e-3;
    *rate_hz = window_s > 0.0 ? h[0] / (double)n / window_s : 0.0;
    *isi_cv = h[2] > 0.0 ? h[1] / h[2] : 0.0;
    return SNN_OK;
}
