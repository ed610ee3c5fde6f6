// snn_persistent.cuh -- many timesteps in one launch.
//
// For small networks a timestep is a few microseconds of work spread over
// two or three kernel launches, and the launches themselves (the drain of
// one kernel and the ramp of the next, even inside a CUDA graph) take most
// of the step.  Here one cooperative launch runs n steps of the pipeline of
// Fig. 1 (Section III-A-1) with its stages as phases of a loop, separated
// by a grid-wide barrier:
//
//   Update Neurons (every neuron of the batch, a grid-stride loop over the
//   update's 8- or 4-neuron thread groups, with the previous step's
//   bookkeeping) -> barrier -> Receive Spikes of S_{t-d+1} (the global form:
//   rows in pieces over the grid's warps, red.global.add) -> barrier.
//
// The phases are the separate kernels' device functions, so the results are
// theirs bit for bit.  The barrier is a counter and a generation word in
// global memory; every wait is bounded (snn_config.wait_polls polls, default
// kPersistSpin): a CTA whose wait runs out sets kErrTimeout and leaves the
// step loop, after which the barriers of the other CTAs run out too (the
// count they wait for is never reached) and the launch ends.
#pragma once
#include <cuda_runtime.h>

#include "snn_device.cuh"
#include "snn_kernels.cuh"

namespace snn {

constexpr uint32_t kPersistSpin = 1u << 22;  // polls of one barrier wait (each after a 64 ns sleep)

__device__ __forceinline__ uint32_t ld_acquire_u32(const unsigned int* p)
{
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Grid-wide barrier over gridDim.x CTAs (all resident: cooperative launch).
// bar[0]: arrivals of the current generation, bar[1]: the generation.
// Returns false when the bounded wait ran out (kErrTimeout is set).
__device__ __forceinline__ bool grid_barrier(unsigned int* bar, uint32_t spin, Ctl* ctl)
{
    __shared__ uint32_t s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        bool ok = true;
        const uint32_t gen = ld_acquire_u32(bar + 1);
        __threadfence();  // this CTA's writes before its arrival
        if (atomicAdd(bar, 1u) == gridDim.x - 1) {
            bar[0] = 0;
            __threadfence();
            atomicAdd(bar + 1, 1u);  // release the others
        } else {
            uint32_t i = 0;
            while (ld_acquire_u32(bar + 1) == gen) {
                if (++i > spin) {
                    atomicOr(&ctl->err, kErrTimeout);
                    ok = false;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok ? 1u : 0u;
    }
    __syncthreads();
    return s_ok != 0;
}

// n steps from ctl->t; CTA 0 advances ctl->t at the end.  MODEL: 0 Vogels,
// 1 Brunel (no plasticity); W16 / ROWW: the global receive's edge layout.
template <int MODEL, bool W16, bool ROWW, bool STATS, int NPT>
__global__ void __launch_bounds__(256) k_persistent(Net n, uint32_t steps, unsigned int* bar, uint32_t spin)
{
    const unsigned long long t0 = n.ctl->t;
    const uint32_t gid = blockIdx.x * blockDim.x + threadIdx.x, nthreads = gridDim.x * blockDim.x;
    const uint32_t G = n.Np / NPT;
    uint32_t s = 0;
    for (; s < steps; ++s) {
        const unsigned long long t = t0 + s;
        for (uint32_t gt = gid; gt < max(n.n_inst, 1u); gt += nthreads) step_bookkeeping(n, t, gt, false);
        for (uint32_t g0 = 0; g0 < G; g0 += nthreads) update_neurons<MODEL, 0, STATS, NPT>(n, t, g0 + gid, n.acc0);
        if (!grid_barrier(bar, spin, n.ctl)) break;
        receive_global<W16, ROWW>(n, t);
        if (!grid_barrier(bar, spin, n.ctl)) break;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) n.ctl->t = t0 + s;
}

}  // namespace snn
