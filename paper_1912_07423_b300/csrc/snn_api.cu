// snn_api.cu -- host side of the libsnn C ABI (include/snn.h).
//
// The context owns the device arrays described in snn_device.cuh.  A
// timestep is a fixed sequence of kernel launches that read the step index
// from the device control block, so the sequence is captured once into a
// CUDA graph (several steps per graph) and replayed by snn_step.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "../../include/snn.h"
#include "snn_device.cuh"
#include "snn_kernels.cuh"
#include "snn_tiled.cuh"
#include "snn_bulk.cuh"
#include "snn_models.cuh"
#include "snn_fused.cuh"
#include "snn_persistent.cuh"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

using namespace snn;

struct snn_ctx {
    snn_config cfg{};
    std::vector<snn_params> params;
    snn_device dev{};
    cudaStream_t stream = nullptr;   // user stream (may be the legacy default)
    cudaStream_t cap_stream = nullptr;
    cudaStream_t side = nullptr;       // the per-step plan, beside the update when the delay allows
    int plan_priority = 0;             // the greatest stream priority: the plan's block goes before the update's
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    std::string err;

    // sizes and host mirrors of the layout
    uint32_t N = 0, Np = 0, D = 0;
    uint64_t E = 0;
    std::vector<uint32_t> g_off;   // global instance offsets (n_inst+1)
    std::vector<uint32_t> pbase;   // padded bases (n_inst+1)
    std::vector<unsigned long long> log_lo, log_n;  // each instance's region of the raster log
    bool vogels = false, stdp = false, w16 = false, stats = false;
    bool lazy = false;             // lazy Update Synapses (SNN_F_LAZY)
    bool generic = false;          // a model of the generic update (snn_models.cuh)
    int npt = kUpdateNeurons;      // neurons per thread of the fixed models' update
    void* mstate = nullptr;        // generic models: one state record per neuron slot
    size_t mbytes = 0;             // bytes of one record
    bool graph_loaded = false;
    uint64_t host_steps = 0;       // steps enqueued since reset

    // device allocations
    struct Alloc {
        void* p;
        size_t bytes;
    };
    std::vector<Alloc> allocs;
    size_t bytes_held = 0;

    Net net{};
    Ctl* ctl = nullptr;
    uint32_t cr = 0;               // count-ring length
    bool rows_sorted = true;
    InstDev* inst = nullptr;
    uint32_t* inst_of_w32 = nullptr;
    uint4* wdesc = nullptr;
    uint32_t* pois = nullptr;
    uint8_t* pois_start = nullptr;
    uint64_t* roff = nullptr;
    uint32_t* tgt = nullptr;
    int16_t* w16p = nullptr;
    float* w32p = nullptr;
    int32_t* w_init = nullptr;     // weights at load time (lattice), for snn_reset with STDP
    uint8_t* meta = nullptr;
    uint64_t* coff = nullptr;
    uint32_t* cedge = nullptr;
    uint32_t* cpre = nullptr;
    TiledPlan tiled{};
    bool use_tiled = false;
    bool use_bulk = false;             // tiled plan, bulk-copy kernel
    bool packed = false;               // the tiled receive reads pk32
    uint32_t* pk32 = nullptr;          // packed edges: (target - instance base) << 16 | int16 code
    uint16_t* pk16 = nullptr;          // 16-bit target offsets (rows with one weight each)
    bool off16 = false;                // the tiled receive reads pk16 and the row weights
    uint32_t tune_count = 0;           // re-plans done (at most 2)
    uint64_t tune_next = 0;            // step of the next re-plan
    std::vector<unsigned long long> spk_seen;  // instance spike counts at the last re-plan
    std::vector<uint64_t> inst_edges;  // synapses of each instance
    uint4* rinfo = nullptr;            // row records (start, length, meta)
    int32_t* roww = nullptr;           // row weights (16-bit codes, one per row); net.roww points here when used
    // receive form in use (RecvForm) and, with SNN_RECV_AUTO, the ms per step
    // each form took in the tuning run (0: not a candidate)
    int form = 0;
    bool tiled_fits = false;           // every row's length fits its 32-bit row record
    float tune_ms[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
    // persistent multi-step launch (snn_persistent.cuh)
    bool persistent = false;
    uint32_t persist_grid = 0;         // CTAs of 256 threads (all resident)
    uint32_t persist_max = 0;          // the most that are resident at once
    unsigned int* persist_bar = nullptr;  // grid barrier: arrivals, generation
    bool tuned = false;
    // fused step (snn_fused.cuh): update and receive of a step in one kernel
    bool fused = false;
    StepPlan plan2{};                  // the second per-step plan (odd steps)
    uint32_t fused_grid = 0;           // CTAs of the fused kernel (all resident)
    uint32_t fused_lead = 0;           // receive items before update chunks alternate with them
    size_t fused_smem = 0;

    // pinned staging ring of the large host copies (snn_build_graph's upload,
    // snn_read_spikes' readout), allocated at the first one and kept
    static constexpr int kStageBufs = 4;
    static constexpr size_t kStageChunk = 64u << 20;
    void* stage[kStageBufs] = {};
    cudaEvent_t stage_ev[kStageBufs] = {};

    // CUDA graphs: one step, and steps_per_graph steps
    cudaGraphExec_t g1 = nullptr, gk = nullptr;
    uint32_t k_steps = 0;
    uint32_t lazy_blocks = 0;          // grid of the lazy replay: the blocks resident at once
};

namespace {

snn_status fail(snn_ctx* c, snn_status s, const char* fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

#define CUDA_TRY(c, call)                                                                         \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess) return fail(c, SNN_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
    } while (0)

void* dev_alloc(snn_ctx* c, size_t bytes)
{
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~size_t(255);
    void* p = nullptr;
    if (c->dev.alloc) {
        p = c->dev.alloc(bytes, c->dev.stream, c->dev.user);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        c->allocs.push_back({p, bytes});
        c->bytes_held += bytes;
    }
    return p;
}

void dev_free(snn_ctx* c, void* p)
{
    if (!p) return;
    for (size_t i = 0; i < c->allocs.size(); ++i)
        if (c->allocs[i].p == p) {
            c->bytes_held -= c->allocs[i].bytes;
            c->allocs.erase(c->allocs.begin() + i);
            if (c->dev.free)
                c->dev.free(p, c->dev.stream, c->dev.user);
            else
                cudaFree(p);
            return;
        }
}

template <class T>
T* alloc_n(snn_ctx* c, size_t n)
{
    return static_cast<T*>(dev_alloc(c, n * sizeof(T)));
}

// Poisson thresholds T_k = floor(CDF(k) * 2^32) while below 2^32 - 1, with
// the CDF summed from p_k = p_{k-1} * lambda / k in binary64.
int poisson_table(double lambda, uint32_t* T, int cap)
{
    double p = std::exp(-lambda);
    double cdf = p;
    int n = 0;
    for (int k = 0; k < 1000000; ++k) {
        if (k > 0) {
            p = p * lambda / (double)k;
            cdf = cdf + p;
        }
        const double s = std::floor(cdf * 4294967296.0);
        if (s >= 4294967295.0) return n;
        if (n == cap) return -1;
        T[n++] = (uint32_t)s;
    }
    return -1;
}

InstDev make_inst(const snn_params& p, uint32_t pbase, uint32_t goff, uint32_t pois_off, int pois_n)
{
    InstDev d{};
    d.pbase = pbase;
    d.goff = goff;
    d.n = p.n;
    d.n_exc = p.n_exc;
    d.R = p.refractory_steps;
    d.jext = p.jext_q;
    d.wmax = p.w_max_q;
    d.pois_off = pois_off;
    d.pois_n = (uint32_t)pois_n;
    d.Pm = (float)std::exp(-p.dt / p.tau_m);
    d.Pe = (float)(p.tau_e > 0 ? std::exp(-p.dt / p.tau_e) : 0.0);
    d.Pi = (float)(p.tau_i > 0 ? std::exp(-p.dt / p.tau_i) : 0.0);
    d.Pp = (float)(p.tau_plus > 0 ? std::exp(-p.dt / p.tau_plus) : 0.0);
    d.Pn = (float)(p.tau_minus > 0 ? std::exp(-p.dt / p.tau_minus) : 0.0);
    d.Ap = (float)(p.a_plus * (double)p.w_max_q);
    d.Am = (float)(p.a_minus * (double)p.w_max_q);
    d.v_th = (float)p.v_th;
    d.v_reset = (float)p.v_reset;
    d.e_l = (float)p.e_l;
    d.v0_lo = (float)p.v0_lo;
    d.v0_span = (float)p.v0_span;
    return d;
}

uint32_t grid_for(uint64_t threads, uint32_t block) { return (uint32_t)std::max<uint64_t>(1, (threads + block - 1) / block); }

int sm_count()
{
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// k_update<MODEL, SYN, STATS, npt> on Np slots
template <int MODEL, int SYN>
void launch_update(const Net& n, bool stats, int npt, uint32_t Np, cudaStream_t s)
{
    if (npt == kUpdateNeuronsSmall) {
        const uint32_t blocks = grid_for(Np / kUpdateNeuronsSmall, 256);
        if (stats)
            k_update<MODEL, SYN, true, kUpdateNeuronsSmall><<<blocks, 256, 0, s>>>(n);
        else
            k_update<MODEL, SYN, false, kUpdateNeuronsSmall><<<blocks, 256, 0, s>>>(n);
    } else {
        const uint32_t blocks = grid_for(Np / kUpdateNeurons, 256);
        if (stats)
            k_update<MODEL, SYN, true, kUpdateNeurons><<<blocks, 256, 0, s>>>(n);
        else
            k_update<MODEL, SYN, false, kUpdateNeurons><<<blocks, 256, 0, s>>>(n);
    }
}

// The kernels of one timestep, in pipeline order (Fig. 1).  ev, if given,
// holds kPhases + 1 events recorded between the phases.
constexpr int kPhases = 6;

// The edge layout the tiled receive reads.
int recv_wm(const snn_ctx* c)
{
    return c->off16 ? kWOff16 : (c->packed ? kWPacked : (c->w16 ? kW16 : kWF32));
}

FusedDev fused_args(const snn_ctx* c)
{
    FusedDev F{};
    F.tiles = c->tiled.tiles;
    F.split = c->tiled.split;
    F.plan[0] = c->tiled.step;
    F.plan[1] = c->plan2;
    F.n_tiles = c->tiled.n_tiles;
    F.max_len = c->tiled.max_len;
    F.n_ctas = c->fused_grid;
    F.cap = std::min<uint32_t>(kMaxParts, c->fused_grid);
    F.items_cap = c->tiled.items_cap;
    F.n_chunks = (c->Np + kFusedChunk - 1) / kFusedChunk;
    F.lead = c->fused_lead;
    uint32_t n_pad = 1;
    while (n_pad < c->tiled.n_tiles) n_pad <<= 1;
    F.plan_bytes = (uint32_t)plan_smem(n_pad);
    return F;
}

cudaError_t launch_fused(const snn_ctx* c, const Net& n, cudaStream_t s)
{
    const FusedDev F = fused_args(c);
    const dim3 grid(c->fused_grid), block(kFusedThreads);
    if (c->off16) {
        if (c->stats)
            k_step_fused<kWOff16, true><<<grid, block, c->fused_smem, s>>>(n, F);
        else
            k_step_fused<kWOff16, false><<<grid, block, c->fused_smem, s>>>(n, F);
    } else if (c->packed) {
        if (c->stats)
            k_step_fused<kWPacked, true><<<grid, block, c->fused_smem, s>>>(n, F);
        else
            k_step_fused<kWPacked, false><<<grid, block, c->fused_smem, s>>>(n, F);
    } else {
        if (c->stats)
            k_step_fused<kW16, true><<<grid, block, c->fused_smem, s>>>(n, F);
        else
            k_step_fused<kW16, false><<<grid, block, c->fused_smem, s>>>(n, F);
    }
    return cudaGetLastError();
}

snn_status enqueue_step(snn_ctx* c, cudaStream_t s, cudaEvent_t* ev = nullptr, uint32_t k = 0)
{
    Net n = c->net;
    n.k = k;  // step = ctl->t + k
    if (c->fused) {  // update and receive of the step in one kernel (phase [3])
        if (ev)
            for (int i = 0; i <= 3; ++i) cudaEventRecord(ev[i], s);
        CUDA_TRY(c, launch_fused(c, n, s));
        if (ev) {
            cudaEventRecord(ev[4], s);
            cudaEventRecord(ev[5], s);
            k_advance<<<1, 1, 0, s>>>(c->ctl, 1);
            cudaEventRecord(ev[6], s);
        }
        CUDA_TRY(c, cudaGetLastError());
        return SNN_OK;
    }
    if (ev) cudaEventRecord(ev[0], s);
    const uint32_t ublocks = grid_for(c->Np / kUpdateNeurons, 256);
    const uint32_t wblocks = (uint32_t)sm_count() * 8;
    // the tiled receive's plan reads the spike counts of step t + 1 - d: with
    // d >= 2 they are final before this step's update, and the plan runs
    // beside it (after the previous step's merge, which read the last plan)
    const bool planned = c->use_tiled && !c->use_bulk;
    const bool fork = planned && c->cfg.delay >= 2;
    if (fork) {
        CUDA_TRY(c, cudaEventRecord(c->ev_fork, s));
        CUDA_TRY(c, cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        CUDA_TRY(c, enqueue_tiled_plan(c->tiled, n, c->side, c->plan_priority));
        CUDA_TRY(c, cudaEventRecord(c->ev_join, c->side));
    }
    // eager plasticity: depression before the update, potentiation after it;
    // lazy: one replay pass after the update over the transmitting and the
    // expiring rows
    if (c->stdp && !c->lazy) {
        if (c->w16)
            k_stdp_depress<true><<<wblocks, 256, 0, s>>>(n);
        else
            k_stdp_depress<false><<<wblocks, 256, 0, s>>>(n);
    }
    if (ev) cudaEventRecord(ev[1], s);
    if (c->generic)
        launch_update_model(c->cfg.model, n, c->mstate, c->stats, ublocks, s);
    else if (c->vogels)
        launch_update<0, 0>(n, c->stats, c->npt, c->Np, s);
    else if (c->lazy)
        launch_update<1, 2>(n, c->stats, c->npt, c->Np, s);
    else if (c->stdp)
        launch_update<1, 1>(n, c->stats, c->npt, c->Np, s);
    else
        launch_update<1, 0>(n, c->stats, c->npt, c->Np, s);
    if (ev) cudaEventRecord(ev[2], s);
    if (c->lazy) {
        if (c->w16)
            k_stdp_lazy<true><<<c->lazy_blocks, kLazyThreads, 0, s>>>(n);
        else
            k_stdp_lazy<false><<<c->lazy_blocks, kLazyThreads, 0, s>>>(n);
    } else if (c->stdp) {
        if (c->w16)
            k_stdp_potentiate<true><<<wblocks, 256, 0, s>>>(n);
        else
            k_stdp_potentiate<false><<<wblocks, 256, 0, s>>>(n);
    }
    if (ev) cudaEventRecord(ev[3], s);
    cudaEvent_t mid = ev ? ev[4] : nullptr;  // between the receive and the merge
    if (c->use_tiled && c->use_bulk) {
        CUDA_TRY(c, enqueue_bulk_receive(c->tiled, n, c->w16, s, c->cfg.wait_polls ? c->cfg.wait_polls : kBulkSpin, mid));
    } else if (c->use_tiled) {
        if (fork)
            CUDA_TRY(c, cudaStreamWaitEvent(s, c->ev_join, 0));
        else
            CUDA_TRY(c, enqueue_tiled_plan(c->tiled, n, s));
        // with the plan beside the update and no plasticity in between, the
        // receive follows the update as its programmatic dependent
        CUDA_TRY(c, enqueue_tiled_receive(c->tiled, n, recv_wm(c), s,
                                          fork && !c->stdp && !ev));
        if (mid) cudaEventRecord(mid, s);  // no merge: the parts add into the accumulators
    } else {
        if (c->w16 && c->net.roww)
            k_receive_global<true, true><<<wblocks, 256, 0, s>>>(n);
        else if (c->w16)
            k_receive_global<true, false><<<wblocks, 256, 0, s>>>(n);
        else
            k_receive_global<false, false><<<wblocks, 256, 0, s>>>(n);
        if (mid) cudaEventRecord(mid, s);
    }
    if (ev) cudaEventRecord(ev[5], s);
    if (ev) {  // profiled steps run one at a time
        k_advance<<<1, 1, 0, s>>>(c->ctl, 1);
        cudaEventRecord(ev[6], s);
    }
    CUDA_TRY(c, cudaGetLastError());
    return SNN_OK;
}

snn_status capture(snn_ctx* c, uint32_t steps, cudaGraphExec_t* out)
{
    cudaGraph_t g = nullptr;
    CUDA_TRY(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    snn_status st = SNN_OK;
    for (uint32_t i = 0; i < steps && st == SNN_OK; ++i) st = enqueue_step(c, c->cap_stream, nullptr, i);
    if (st == SNN_OK) {
        k_advance<<<1, 1, 0, c->cap_stream>>>(c->ctl, steps);
        if (cudaGetLastError() != cudaSuccess) st = fail(c, SNN_E_CUDA, "graph capture: k_advance launch");
    }
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (st != SNN_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(out, g, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    return SNN_OK;
}

void drop_graphs(snn_ctx* c)
{
    if (c->g1) cudaGraphExecDestroy(c->g1);
    if (c->gk) cudaGraphExecDestroy(c->gk);
    c->g1 = c->gk = nullptr;
}

snn_status check_device_errors(snn_ctx* c)
{
    unsigned int err = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&err, &c->ctl->err, sizeof err, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (err & kErrTimeout) return fail(c, SNN_E_TIMEOUT, "a bounded device-side wait gave up");
    if (err & kErrPlan) return fail(c, SNN_E_OVERFLOW, "the receive plan of a step did not fit its buffer");
    if (err & kErrLazyAge) return fail(c, SNN_E_STATE, "a lazily updated row outlived its spike history");
    if (err & kErrLogOverflow)
        return fail(c, SNN_E_OVERFLOW, "the spike log is full (an instance filled its share of log_capacity = %llu)",
                    (unsigned long long)c->cfg.log_capacity);
    return SNN_OK;
}

// Lazy plasticity: bring every stale row up to date after the last step,
// before the weights or the presynaptic traces are read or written.
snn_status lazy_flush(snn_ctx* c)
{
    if (!c->lazy) return SNN_OK;
    unsigned long long t = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&t, &c->ctl->t, sizeof t, cudaMemcpyDeviceToHost, c->stream));
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (t == 0) return SNN_OK;
    Net n = c->net;
    n.k = 0;
    const uint32_t blocks = (uint32_t)sm_count() * 8;
    if (c->w16)
        k_stdp_flush<true><<<blocks, 256, 0, c->stream>>>(n, t - 1);
    else
        k_stdp_flush<false><<<blocks, 256, 0, c->stream>>>(n, t - 1);
    CUDA_TRY(c, cudaGetLastError());
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNN_OK;
}

snn_status init_state(snn_ctx* c)
{
    k_init_state<<<grid_for(c->Np / 4, 256), 256, 0, c->stream>>>(c->net, c->vogels ? 1 : 0, c->stdp ? 1 : 0,
                                                                   c->lazy ? 1 : 0);
    CUDA_TRY(c, cudaGetLastError());
    if (c->generic) {
        launch_init_model(c->cfg.model, c->net, c->mstate, grid_for(c->Np / 8, 256), c->stream);
        CUDA_TRY(c, cudaGetLastError());
    }
    if (c->lazy) {
        CUDA_TRY(c, cudaMemsetAsync(c->net.xcount, 0, 2 * sizeof(unsigned int), c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->net.hist, 0, (size_t)c->Np * 2 * sizeof(unsigned long long), c->stream));
    }
    // control block: step 0, empty queues and log
    CUDA_TRY(c, cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->stream));
    if (c->stdp)
        CUDA_TRY(c, cudaMemsetAsync(c->net.bits, 0, (size_t)c->D * (c->Np / 32) * sizeof(uint32_t), c->stream));
    if (c->stats) {
        CUDA_TRY(c, cudaMemsetAsync(c->net.st_cnt, 0, (size_t)c->Np * 4, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->net.st_sum, 0, (size_t)c->Np * 8, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->net.st_sq, 0, (size_t)c->Np * 8, c->stream));
    }
    CUDA_TRY(c, cudaMemsetAsync(c->net.icount, 0, (size_t)c->cr * c->cfg.n_inst * 4, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->net.ilog, 0, 2 * (size_t)c->cfg.n_inst * 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->net.inst_spikes, 0, (size_t)c->cfg.n_inst * 8, c->stream));
    CUDA_TRY(c, cudaMemsetAsync(c->net.tile_ctr, 0, 2 * sizeof(unsigned int), c->stream));
    if (c->persist_bar) CUDA_TRY(c, cudaMemsetAsync(c->persist_bar, 0, 2 * sizeof(unsigned int), c->stream));
    if (c->fused) {  // the input of step 1 and the plans of steps 0 and 1
        CUDA_TRY(c, cudaMemsetAsync(c->net.accx, 0, (size_t)c->Np * 4, c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->tiled.step.hdr, 0, 4 * sizeof(uint32_t), c->stream));
        CUDA_TRY(c, cudaMemsetAsync(c->plan2.hdr, 0, 4 * sizeof(uint32_t), c->stream));
    }
    c->host_steps = 0;
    return SNN_OK;
}

// The tiled receive can read packed edges: int16 codes, no plasticity, every
// instance's offsets within 16 bits, and the caller did not opt out.
bool packable(const snn_ctx* c)
{
    if (c->use_bulk || !c->w16 || c->stdp || (c->cfg.flags & SNN_F_UNPACKED)) return false;
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b)
        if (c->pbase[b + 1] - c->pbase[b] > 65536u) return false;
    return true;
}

// (Re)build the packed edges from the target and code arrays.
// Row weights for the global receive: with 16-bit codes and no plasticity
// (and no SNN_F_UNPACKED), a graph whose every row carries one weight -- the
// source population's, as in the paper's models -- keeps it per row and the
// receive reads 4 bytes per event.  Recomputed after snn_write_state(W); the
// CUDA graphs are re-captured when the layout changes.
snn_status refresh_row_weights(snn_ctx* c, bool* changed)
{
    *changed = false;
    const int32_t* before = c->net.roww;
    c->net.roww = nullptr;
    if (c->w16 && !c->stdp && !(c->cfg.flags & SNN_F_UNPACKED)) {
        if (!c->roww) c->roww = alloc_n<int32_t>(c, c->Np);
        unsigned int* dmixed = alloc_n<unsigned int>(c, 1);
        if (!c->roww || !dmixed) {
            dev_free(c, dmixed);
            return fail(c, SNN_E_NOMEM, "row weights");
        }
        unsigned int mixed = 0;
        cudaError_t e = cudaMemsetAsync(dmixed, 0, 4, c->stream);
        if (e == cudaSuccess) {
            k_row_weights<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->roff, c->w16p, c->meta, c->Np, c->roww,
                                                                             dmixed);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&mixed, dmixed, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, dmixed);
        if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "row weights: %s", cudaGetErrorString(e));
        if (!mixed) c->net.roww = c->roww;
    }
    *changed = (before != nullptr) != (c->net.roww != nullptr);
    return SNN_OK;
}

// 16-bit target offsets apply where packed edges do and every row carries
// one weight (the row weights are in use).
bool off16able(const snn_ctx* c) { return packable(c) && c->net.roww != nullptr; }

snn_status pack_off16(snn_ctx* c)
{
    if (!c->off16) return SNN_OK;
    k_pack_off16<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->net, c->Np, c->pk16);
    CUDA_TRY(c, cudaGetLastError());
    return SNN_OK;
}

snn_status pack_edges(snn_ctx* c)
{
    if (!c->packed) return SNN_OK;
    k_pack_edges<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->net, c->Np, c->pk32);
    CUDA_TRY(c, cudaGetLastError());
    return SNN_OK;
}

// The context's pinned staging ring, allocated at its first use.
snn_status stage_ring(snn_ctx* c)
{
    for (int i = 0; i < snn_ctx::kStageBufs; ++i) {
        if (!c->stage[i] && cudaHostAlloc(&c->stage[i], snn_ctx::kStageChunk, cudaHostAllocDefault) != cudaSuccess) {
            c->stage[i] = nullptr;
            return fail(c, SNN_E_CUDA, "pinned staging buffers");
        }
        if (!c->stage_ev[i] && cudaEventCreateWithFlags(&c->stage_ev[i], cudaEventDisableTiming) != cudaSuccess) {
            c->stage_ev[i] = nullptr;
            return fail(c, SNN_E_CUDA, "staging events");
        }
    }
    return SNN_OK;
}

// Host threads that copy one chunk together, each its stripe: started once
// per staged transfer and reused for every chunk (starting threads per chunk
// cost about 1.5 ms for 16 on the hosts measured, as much as copying a
// 64 MB chunk).  copy() returns when the whole chunk is copied; the workers
// spin between chunks and leave when the copier is destroyed.
class StripeCopier {
  public:
    explicit StripeCopier(unsigned nth)
    {
        // as many workers as the host lets us start (the caller copies stripe 0)
        try {
            workers_.reserve(nth);
            for (unsigned t = 1; t < std::max(1u, nth); ++t) workers_.emplace_back([this, t]() { work(t); });
        } catch (...) {
        }
        nth_ = (unsigned)workers_.size() + 1;
    }
    ~StripeCopier()
    {
        quit_.store(true, std::memory_order_release);
        for (auto& th : workers_) th.join();
    }
    void copy(char* to, const char* from, size_t len)
    {
        to_ = to;
        from_ = from;
        len_ = len;
        part_ = (len / nth_ + 63) & ~size_t(63);
        done_.store(0, std::memory_order_relaxed);
        gen_.fetch_add(1, std::memory_order_release);
        stripe(0);
        while (done_.load(std::memory_order_acquire) != nth_ - 1) std::this_thread::yield();
    }

  private:
    void stripe(unsigned t)
    {
        const size_t b = (size_t)t * part_;
        if (b < len_) std::memcpy(to_ + b, from_ + b, std::min(part_, len_ - b));
    }
    void work(unsigned t)
    {
        uint64_t seen = 0;
        for (;;) {
            uint64_t g;
            while ((g = gen_.load(std::memory_order_acquire)) == seen) {
                if (quit_.load(std::memory_order_acquire)) return;
                std::this_thread::yield();
            }
            seen = g;
            stripe(t);
            done_.fetch_add(1, std::memory_order_release);
        }
    }
    std::atomic<unsigned> nth_{1};
    std::vector<std::thread> workers_;
    std::atomic<uint64_t> gen_{0};
    std::atomic<unsigned> done_{0};
    std::atomic<bool> quit_{false};
    char* to_ = nullptr;
    const char* from_ = nullptr;
    size_t len_ = 0, part_ = 0;
};

unsigned stage_threads()
{
    const unsigned hw = std::thread::hardware_concurrency();
    return std::max(1u, std::min(16u, hw ? hw : 1u));
}

// Host -> device copy of a large pageable array: chunks are copied into the
// pinned ring by several host threads while the DMA engine moves the
// previous chunks (the driver's own staging of pageable memory copies with
// one thread).  Waits for the stream.
snn_status upload(snn_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    constexpr size_t kChunk = snn_ctx::kStageChunk;
    constexpr int kBufs = snn_ctx::kStageBufs;
    if (bytes <= kChunk) {
        CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s));
        return SNN_OK;
    }
    snn_status st = stage_ring(c);
    void** buf = c->stage;
    cudaEvent_t* done = c->stage_ev;
    StripeCopier copier(stage_threads());
    for (size_t off = 0, i = 0; off < bytes && st == SNN_OK; off += kChunk, i = (i + 1) % kBufs) {
        const size_t len = std::min(kChunk, bytes - off);
        if (cudaEventSynchronize(done[i]) != cudaSuccess) {
            st = fail(c, SNN_E_CUDA, "staging wait");
            break;
        }
        copier.copy(static_cast<char*>(buf[i]), static_cast<const char*>(src) + off, len);
        if (cudaMemcpyAsync(static_cast<char*>(dst) + off, buf[i], len, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaEventRecord(done[i], s) != cudaSuccess)
            st = fail(c, SNN_E_CUDA, "staged copy");
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SNN_OK) st = fail(c, SNN_E_CUDA, "staged copy");
    return st;
}

// Device -> host copy into a large pageable array, the reverse of upload():
// the DMA engine fills a ring of pinned buffers ahead while several host
// threads copy the filled ones out (and take the page faults of a fresh
// destination in parallel).  Waits for the stream.
snn_status download(snn_ctx* c, void* dst, const void* src, size_t bytes, cudaStream_t s)
{
    constexpr size_t kChunk = snn_ctx::kStageChunk;
    constexpr int kBufs = snn_ctx::kStageBufs;
    if (bytes <= kChunk) {
        CUDA_TRY(c, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s));
        CUDA_TRY(c, cudaStreamSynchronize(s));
        return SNN_OK;
    }
    snn_status st = stage_ring(c);
    void** buf = c->stage;
    cudaEvent_t* full = c->stage_ev;
    const size_t n = (bytes + kChunk - 1) / kChunk;
    auto fetch = [&](size_t k) {
        const size_t off = k * kChunk, len = std::min(kChunk, bytes - off);
        if (cudaMemcpyAsync(buf[k % kBufs], static_cast<const char*>(src) + off, len, cudaMemcpyDeviceToHost, s) !=
                cudaSuccess ||
            cudaEventRecord(full[k % kBufs], s) != cudaSuccess)
            st = fail(c, SNN_E_CUDA, "staged copy");
    };
    for (size_t k = 0; k < n && k < (size_t)kBufs && st == SNN_OK; ++k) fetch(k);
    StripeCopier copier(stage_threads());
    for (size_t k = 0; k < n && st == SNN_OK; ++k) {
        if (cudaEventSynchronize(full[k % kBufs]) != cudaSuccess) {
            st = fail(c, SNN_E_CUDA, "staging wait");
            break;
        }
        const size_t off = k * kChunk, len = std::min(kChunk, bytes - off);
        copier.copy(static_cast<char*>(dst) + off, static_cast<const char*>(buf[k % kBufs]), len);
        if (k + kBufs < n) fetch(k + kBufs);
    }
    if (cudaStreamSynchronize(s) != cudaSuccess && st == SNN_OK) st = fail(c, SNN_E_CUDA, "staged copy");
    return st;
}

// Cut the tiles of the tiled receive; work[b] = expected delivered edges of
// instance b per step (null: proportional to its synapses).
snn_status plan_tiles(snn_ctx* c, const double* work)
{
    // accumulators of one tile: 112 KB (tiled, two CTAs per SM), or what the
    // copy ring leaves of the 227 KB (bulk, one CTA per SM)
    const uint32_t ch = c->vogels ? 2u : 1u;
    const uint32_t bulk_len = (uint32_t)((227u * 1024u - 1024u - kBulkSlots * bulk_slot_bytes(c->w16)) / 4u / 256u * 256u);
    const uint32_t max_len = (c->use_bulk ? bulk_len : kTiledMaxWords) / ch / 256u * 256u;
    const int wm = off16able(c) ? kWOff16 : (packable(c) ? kWPacked : (c->w16 ? kW16 : kWF32));
    // row segments are cut into pieces only from 1.5 piece_edges up (1,536 edges at 2 bytes per edge,
    // 2,304 packed): on the sweep pieces from 768 edges cost 0.5 % of the step, from 384 edges 17 %
    snn_status st = tiled_plan(c->tiled, c->net, c->params.data(), c->pbase.data(), c->cfg.n_inst, (int)ch, max_len,
                               work, c->inst_edges.data(), sm_count(), [c](size_t b) { return dev_alloc(c, b); },
                               [c](void* p) { dev_free(c, p); }, c->stream, !c->use_bulk, 256u * vec_of(wm));
    if (st == SNN_OK && c->use_bulk) {
        int dev = 0, optin = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        const size_t smem = bulk_smem(c->tiled.max_len, (int)ch, c->w16);
        if (smem > (size_t)optin) return SNN_E_ARG;
        if (bulk_set_smem(smem) != cudaSuccess) return SNN_E_CUDA;
    }
    return st;
}

// Re-cut the tiles by the spikes measured so far (results do not depend on
// the tiling, only the balance across SMs does), then re-capture the graphs.
snn_status retune(snn_ctx* c)
{
    c->tune_count++;
    std::vector<unsigned long long> spk(c->cfg.n_inst, 0);
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    CUDA_TRY(c, cudaMemcpy(spk.data(), c->net.inst_spikes, spk.size() * 8, cudaMemcpyDeviceToHost));
    {  // the last step's counts are folded in by the next update
        unsigned long long t = 0;
        CUDA_TRY(c, cudaMemcpy(&t, &c->ctl->t, 8, cudaMemcpyDeviceToHost));
        if (t > 0) {
            std::vector<unsigned int> last(c->cfg.n_inst, 0);
            CUDA_TRY(c, cudaMemcpy(last.data(), c->net.icount + (size_t)((t - 1) & (c->cr - 1)) * c->cfg.n_inst,
                                   last.size() * 4, cudaMemcpyDeviceToHost));
            for (uint32_t b = 0; b < c->cfg.n_inst; ++b) spk[b] += last[b];
        }
    }
    std::vector<double> work(c->cfg.n_inst, 0.0);
    double total = 0.0;
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b) {
        const double deg = c->params[b].n ? (double)c->inst_edges[b] / c->params[b].n : 0.0;
        // delivered edges plus the fixed work per spike (row record, splits),
        // from the spikes since the previous re-plan
        const unsigned long long d = spk[b] >= c->spk_seen[b] ? spk[b] - c->spk_seen[b] : spk[b];
        work[b] = (double)d * (deg + 8.0);
        total += work[b];
    }
    c->spk_seen = spk;
    if (total <= 0.0) return SNN_OK;
    snn_status st = plan_tiles(c, work.data());
    if (st != SNN_OK) return fail(c, st, "re-cutting the tiles failed");
    drop_graphs(c);
    st = capture(c, 1, &c->g1);
    if (st == SNN_OK && c->k_steps > 1) st = capture(c, c->k_steps, &c->gk);
    return st;
}

// The fused step (snn_fused.cuh) applies to the fixed Brunel model without
// plasticity, the tiled receive with its per-step plan, 16-bit weights and a
// delay of at least 3 steps (the plan of step t+1 made during step t reads
// the spike counts of step t+2-d).
bool fused_applies(const snn_ctx* c)
{
    return c->use_tiled && !c->use_bulk && !c->vogels && !c->generic && !c->stdp && c->w16 && c->cfg.delay >= 3;
}

// Turns the fused step on (its second plan sized like the first, which
// tiled_plan re-allocates with the tiles).  Returns SNN_OK with c->fused
// false when the kernel does not fit.
snn_status setup_fused(snn_ctx* c)
{
    c->fused = false;
    if (!fused_applies(c)) return SNN_OK;
    uint32_t n_pad = 1;
    while (n_pad < c->tiled.n_tiles) n_pad <<= 1;
    const size_t smem = std::max<size_t>((size_t)c->tiled.max_len * 4, plan_smem(n_pad));
    auto set = [&](auto kernel) { return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); };
    if (set(k_step_fused<kWPacked, false>) != cudaSuccess || set(k_step_fused<kWPacked, true>) != cudaSuccess ||
        set(k_step_fused<kW16, false>) != cudaSuccess || set(k_step_fused<kW16, true>) != cudaSuccess ||
        set(k_step_fused<kWOff16, false>) != cudaSuccess || set(k_step_fused<kWOff16, true>) != cudaSuccess) {
        cudaGetLastError();
        return SNN_OK;  // keep the separate kernels
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_step_fused<kWPacked, false>, kFusedThreads, smem) !=
            cudaSuccess ||
        per_sm < 1) {
        cudaGetLastError();
        return SNN_OK;
    }
    c->fused_grid = (uint32_t)(sm_count() * per_sm);
    c->fused_smem = smem;
    c->fused_lead = c->fused_grid;
    dev_free(c, c->plan2.hdr);
    dev_free(c, c->plan2.items);
    dev_free(c, c->plan2.parts);
    c->plan2.hdr = alloc_n<uint32_t>(c, 4);
    c->plan2.items = alloc_n<ItemDev>(c, c->tiled.items_cap);
    c->plan2.parts = alloc_n<uint32_t>(c, c->tiled.n_tiles);
    if (!c->net.accx) c->net.accx = alloc_n<int32_t>(c, c->Np);
    if (!c->plan2.hdr || !c->plan2.items || !c->plan2.parts || !c->net.accx)
        return fail(c, SNN_E_NOMEM, "fused step buffers");
    c->fused = true;
    return SNN_OK;
}

// The receive forms a context can run.  Results do not depend on the form.
enum RecvForm : int { kFormGlobal = 0, kFormTiled = 1, kFormFused = 2, kFormBulk = 3, kFormPersist = 4, kForms = 5 };

// The persistent launch applies to the fixed models without plasticity (its
// receive is the global form).
bool persist_applies(const snn_ctx* c) { return !c->generic && !c->stdp; }

// k_persistent<...> for the context's model and layout, as a function pointer.
void* persist_kernel(const snn_ctx* c)
{
    const bool rw = c->net.roww != nullptr;
#define SNN_PK(M, W, R, S, P) reinterpret_cast<void*>(&k_persistent<M, W, R, S, P>)
#define SNN_PK_NPT(M, W, R, S) (c->npt == kUpdateNeuronsSmall ? SNN_PK(M, W, R, S, kUpdateNeuronsSmall) : SNN_PK(M, W, R, S, kUpdateNeurons))
#define SNN_PK_S(M, W, R) (c->stats ? SNN_PK_NPT(M, W, R, true) : SNN_PK_NPT(M, W, R, false))
#define SNN_PK_W(M) (c->w16 ? (rw ? SNN_PK_S(M, true, true) : SNN_PK_S(M, true, false)) : SNN_PK_S(M, false, false))
    return c->vogels ? SNN_PK_W(0) : SNN_PK_W(1);
#undef SNN_PK_W
#undef SNN_PK_S
#undef SNN_PK_NPT
#undef SNN_PK
}

// n steps in one cooperative launch of c->persist_grid CTAs.
snn_status launch_persistent(snn_ctx* c, uint32_t steps)
{
    if (!steps) return SNN_OK;
    Net n = c->net;
    n.k = 0;
    unsigned int* bar = c->persist_bar;
    uint32_t spin = c->cfg.wait_polls ? c->cfg.wait_polls : kPersistSpin;
    void* args[] = {&n, &steps, &bar, &spin};
    CUDA_TRY(c, cudaLaunchCooperativeKernel(persist_kernel(c), dim3(c->persist_grid), dim3(256), args, 0, c->stream));
    return SNN_OK;
}

// The CTAs a persistent launch can hold at once, and its barrier words.
snn_status setup_persistent(snn_ctx* c)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persist_kernel(c), 256, 0) != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return SNN_E_ARG;
    }
    int dev = 0, coop = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
    if (!coop) return SNN_E_ARG;
    c->persist_max = (uint32_t)(sm_count() * per_sm);
    if (!c->persist_bar) c->persist_bar = alloc_n<unsigned int>(c, 2);
    if (!c->persist_bar) return fail(c, SNN_E_NOMEM, "grid barrier");
    CUDA_TRY(c, cudaMemsetAsync(c->persist_bar, 0, 2 * sizeof(unsigned int), c->stream));
    return SNN_OK;
}

// Grid of a persistent launch: "small" covers the update's thread groups in
// one pass (fewer CTAs: cheaper barriers), else every resident CTA.
uint32_t persist_grid_for(const snn_ctx* c, bool small)
{
    const uint32_t groups = c->Np / (uint32_t)c->npt;
    const uint32_t need = std::max<uint32_t>(1, (groups + 255) / 256);
    return small ? std::min(need, c->persist_max) : c->persist_max;
}

// n steps of the context's form: CUDA graphs, or one persistent launch.
snn_status run_steps(snn_ctx* c, uint32_t n)
{
    if (c->persistent) return launch_persistent(c, n);
    while (c->gk && n >= c->k_steps) {
        CUDA_TRY(c, cudaGraphLaunch(c->gk, c->stream));
        n -= c->k_steps;
    }
    while (n--) CUDA_TRY(c, cudaGraphLaunch(c->g1, c->stream));
    return SNN_OK;
}

// Switches the context to a receive form: builds what it reads (tiles and
// split tables, packed edges, the fused step's buffers), frees the packed
// edges when it does not read them, and captures the step graphs.  The
// neuron state is not touched.  SNN_E_ARG when the form does not fit the
// graph (the context then runs the global receive).
snn_status use_form(snn_ctx* c, int form, uint32_t persist_grid = 0)
{
    drop_graphs(c);
    c->fused = false;
    c->persistent = false;
    c->use_tiled = form != kFormGlobal && form != kFormPersist;
    c->use_bulk = form == kFormBulk;
    snn_status st = SNN_OK;
    if (c->use_tiled) {
        st = (c->rows_sorted && c->tiled_fits) ? plan_tiles(c, nullptr) : SNN_E_ARG;
        if (st == SNN_OK && off16able(c) && !c->pk16) {  // targets only: 2 bytes per edge
            c->pk16 = alloc_n<uint16_t>(c, c->E + 32);
            if (!c->pk16) return fail(c, SNN_E_NOMEM, "16-bit edge offsets");
            CUDA_TRY(c, cudaMemsetAsync(c->pk16, 0, (c->E + 32) * 2, c->stream));
            c->off16 = true;
            c->net.pk16 = c->pk16;
            st = pack_off16(c);
        } else if (st == SNN_OK && !off16able(c) && packable(c) && !c->pk32) {
            c->pk32 = alloc_n<uint32_t>(c, c->E + 16);
            if (!c->pk32) return fail(c, SNN_E_NOMEM, "packed edges");
            CUDA_TRY(c, cudaMemsetAsync(c->pk32, 0, (c->E + 16) * 4, c->stream));
            c->packed = true;
            c->net.pk = c->pk32;
            st = pack_edges(c);
        }
        if (st == SNN_OK && form == kFormFused) {
            st = setup_fused(c);
            if (st == SNN_OK && !c->fused) st = SNN_E_ARG;
        }
    }
    if (st != SNN_OK || !c->use_tiled) {
        tiled_free(c->tiled, [c](void* p) { dev_free(c, p); });
        c->use_tiled = c->use_bulk = c->fused = false;
    }
    c->off16 = c->use_tiled && c->pk16 && off16able(c);
    if (!c->off16 && c->pk16) {
        dev_free(c, c->pk16);
        c->pk16 = nullptr;
    }
    c->net.pk16 = c->off16 ? c->pk16 : nullptr;
    c->packed = c->use_tiled && !c->off16 && c->pk32 && packable(c);
    if (!c->packed && c->pk32) {
        dev_free(c, c->pk32);
        c->pk32 = nullptr;
    }
    c->net.pk = c->packed ? c->pk32 : nullptr;
    if (st == SNN_OK && form == kFormPersist) {
        st = persist_applies(c) ? setup_persistent(c) : SNN_E_ARG;
        if (st == SNN_OK) {
            c->persistent = true;
            c->persist_grid = persist_grid ? std::min(persist_grid, c->persist_max) : persist_grid_for(c, true);
        }
    }
    c->form = c->persistent ? kFormPersist
                            : (c->fused ? kFormFused : (c->use_bulk ? kFormBulk : (c->use_tiled ? kFormTiled : kFormGlobal)));
    if (c->persistent) return SNN_OK;  // no graphs: one launch per snn_step
    snn_status cs = capture(c, 1, &c->g1);
    if (cs == SNN_OK && c->k_steps > 1) cs = capture(c, c->k_steps, &c->gk);
    return st != SNN_OK ? st : cs;
}

// N_0 again: the weights loaded by snn_build_graph (plasticity changes
// them) and the initial neuron state.
snn_status reset_state(snn_ctx* c)
{
    if (c->stdp) {
        k_weights_in<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->roff, c->meta, c->w_init, c->w16 ? 1 : 0,
                                                                        c->Np, c->w16p, c->w32p, &c->ctl->err);
        CUDA_TRY(c, cudaGetLastError());
    }
    return init_state(c);
}

// Steps of a tuning run before its timed window, and in it.
uint32_t tune_warm_steps(const snn_ctx* c) { return std::min<uint32_t>(c->cfg.delay + 150u, 1100u); }
constexpr uint32_t kTuneSteps = 48;
constexpr uint32_t kTuneProbe = 32;   // steps after which a clearly slower form is dropped
constexpr float kTuneAbort = 2.0f;    // ... when its steps took this many times the best so far

// SNN_RECV_AUTO: every form that applies runs from the initial state N_0
// over the same steps (past the first deliveries), timed with CUDA events
// over the last kTuneSteps of them; the fastest is kept.  The simulation is
// deterministic, so every form meets the same spikes; the caller's run
// starts from N_0 afterwards (init_state).  The tiled forms go first; a
// later form whose first kTuneProbe steps already took kTuneAbort times the
// best ms/step so far stops there (its estimate is what snn_info reports).
snn_status tune_receive(snn_ctx* c)
{
    // candidates: (form, persistent grid); the persistent launch twice, with
    // the fewest CTAs that cover the update and with every resident CTA
    int cand[kForms + 1];
    uint32_t cgrid[kForms + 1] = {};
    int nc = 0;
    if (c->rows_sorted && c->tiled_fits) {
        cand[nc++] = kFormTiled;
        c->use_tiled = true;
        c->use_bulk = false;
        if (!(c->cfg.flags & SNN_F_SERIAL) && fused_applies(c)) cand[nc++] = kFormFused;
        c->use_tiled = false;
    }
    cand[nc++] = kFormGlobal;
    if (persist_applies(c) && !(c->cfg.flags & SNN_F_SERIAL) && setup_persistent(c) == SNN_OK) {
        const uint32_t g0 = persist_grid_for(c, true), g1 = persist_grid_for(c, false);
        cand[nc] = kFormPersist;
        cgrid[nc++] = g0;
        if (g1 != g0) {
            cand[nc] = kFormPersist;
            cgrid[nc++] = g1;
        }
    }
    for (float& x : c->tune_ms) x = 0.f;
    if (nc == 1) return use_form(c, cand[0]);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    CUDA_TRY(c, cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return fail(c, SNN_E_CUDA, "cudaEventCreate");
    }
    int best = -1;
    uint32_t best_grid = 0;
    float best_ms = 0.f;
    snn_status st = SNN_OK;
    const uint32_t warm = tune_warm_steps(c);
    auto launch = [&](uint32_t n) -> snn_status { return run_steps(c, n); };
    for (int i = 0; i < nc && st == SNN_OK; ++i) {
        st = use_form(c, cand[i], cgrid[i]);
        if (st == SNN_E_ARG) {  // the form does not fit after all: not a candidate
            st = SNN_OK;
            continue;
        }
        if (st == SNN_OK) st = reset_state(c);
        // a form already kTuneAbort times slower than the best so far over its
        // first kTuneProbe steps is not timed further
        uint32_t left = warm;
        if (st == SNN_OK && best >= 0 && kTuneProbe < warm) {
            float pms = 0.f;
            if (cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, SNN_E_CUDA, "event record");
            if (st == SNN_OK) st = launch(kTuneProbe);
            if (st == SNN_OK && (cudaEventRecord(e1, c->stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                                 cudaEventElapsedTime(&pms, e0, e1) != cudaSuccess))
                st = fail(c, SNN_E_CUDA, "tuning probe");
            if (st == SNN_OK && pms / kTuneProbe > kTuneAbort * best_ms) {
                const float per = pms / kTuneProbe;
                if (c->tune_ms[cand[i]] == 0.f || per < c->tune_ms[cand[i]]) c->tune_ms[cand[i]] = per;
                continue;
            }
            left = warm - kTuneProbe;
        }
        if (st == SNN_OK) st = launch(left);
        if (st == SNN_OK && cudaEventRecord(e0, c->stream) != cudaSuccess) st = fail(c, SNN_E_CUDA, "event record");
        if (st == SNN_OK) st = launch(kTuneSteps);
        if (st == SNN_OK && cudaEventRecord(e1, c->stream) != cudaSuccess) st = fail(c, SNN_E_CUDA, "event record");
        if (st == SNN_OK) {  // a log too small for the tuning steps is no error here: the log starts over
            unsigned int err = 0;
            if (cudaMemcpyAsync(&err, &c->ctl->err, sizeof err, cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
                cudaStreamSynchronize(c->stream) != cudaSuccess)
                st = fail(c, SNN_E_CUDA, "tuning run");
            else if (err & ~kErrLogOverflow)
                st = check_device_errors(c);
        }
        float ms = 0.f;
        if (st == SNN_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) st = fail(c, SNN_E_CUDA, "event time");
        if (st == SNN_OK) {
            const float per = ms / kTuneSteps;
            if (c->tune_ms[cand[i]] == 0.f || per < c->tune_ms[cand[i]]) c->tune_ms[cand[i]] = per;
            if (best < 0 || per < best_ms) {
                best = cand[i];
                best_grid = cgrid[i];
                best_ms = per;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != SNN_OK) return st;
    return use_form(c, best < 0 ? kFormGlobal : best, best_grid);
}

}  // namespace

extern "C" {

const char* snn_status_string(snn_status s)
{
    switch (s) {
    case SNN_OK: return "ok";
    case SNN_E_ARG: return "invalid argument";
    case SNN_E_NOMEM: return "out of memory";
    case SNN_E_CUDA: return "CUDA error";
    case SNN_E_OVERFLOW: return "overflow";
    case SNN_E_TIMEOUT: return "device-side timeout";
    case SNN_E_STATE: return "call out of order";
    }
    return "unknown status";
}

const char* snn_last_error(const snn_ctx* ctx) { return ctx ? ctx->err.c_str() : ""; }

snn_status snn_create(const snn_config* cfg, const snn_params* params, const snn_device* dev, snn_ctx** out)
{
    if (!out) return SNN_E_ARG;
    *out = nullptr;
    if (!cfg || !params || cfg->n_inst == 0) return SNN_E_ARG;
    if (cfg->model > SNN_MODEL_BRUNEL_LIF || cfg->delay < 1 || cfg->delay > 1000) return SNN_E_ARG;
    if ((cfg->flags & SNN_F_STDP) && cfg->model != SNN_BRUNEL) return SNN_E_ARG;
    if ((cfg->flags & SNN_F_LAZY) &&
        (!(cfg->flags & SNN_F_STDP) || cfg->lazy_fifo == 1 || cfg->lazy_fifo > (uint32_t)kLazyMaxF))
        return SNN_E_ARG;
    if (cfg->receive > SNN_RECV_PERSISTENT) return SNN_E_ARG;
    uint64_t N = 0, Np = 0;
    for (uint32_t b = 0; b < cfg->n_inst; ++b) {
        const snn_params& p = params[b];
        if (p.n_exc > p.n || p.refractory_steps > 255) return SNN_E_ARG;
        if (!(p.dt > 0) || !(p.tau_m > 0) || !(p.lambda >= 0)) return SNN_E_ARG;
        if (cfg->model == SNN_VOGELS_CUBA && (!(p.tau_e > 0) || !(p.tau_i > 0))) return SNN_E_ARG;
        if ((cfg->flags & SNN_F_STDP) &&
            (!(p.tau_plus > 0) || !(p.tau_minus > 0) || p.w_max_q < 0 || p.w_max_q > 32767))
            return SNN_E_ARG;
        uint32_t T[kPoissonCap];
        if (cfg->model != SNN_VOGELS_CUBA && poisson_table(p.lambda, T, kPoissonCap) < 0) return SNN_E_ARG;
        N += p.n;
        Np += (p.n + kPad - 1) / kPad * kPad;
    }
    if (Np >= (1ull << 31)) return SNN_E_ARG;

    snn_ctx* c = new (std::nothrow) snn_ctx();
    if (!c) return SNN_E_NOMEM;
    c->cfg = *cfg;
    c->params.assign(params, params + cfg->n_inst);
    if (dev) c->dev = *dev;
    c->stream = (cudaStream_t)c->dev.stream;
    c->vogels = cfg->model == SNN_VOGELS_CUBA;
    c->generic = is_generic_model(cfg->model);
    // 4 neurons per thread for Vogels (its state takes 64 registers at 8 per
    // thread: 4 measured 10 % faster on the 1M-neuron network), and for
    // Brunel when 8 would give fewer 256-thread blocks than SMs (a
    // 100k-neuron network: 49 blocks; 4 % faster there, 8 % slower on the
    // 3.2M-neuron sweep)
    c->npt = (c->vogels || (uint64_t)Np / kUpdateNeurons / 256 < (uint64_t)sm_count()) ? kUpdateNeuronsSmall
                                                                                       : kUpdateNeurons;
    c->mbytes = model_state_bytes(cfg->model);
    c->stdp = (cfg->flags & SNN_F_STDP) != 0;
    c->lazy = c->stdp && (cfg->flags & SNN_F_LAZY) != 0;
    c->w16 = (cfg->flags & SNN_F_W16) != 0;
    c->stats = (cfg->flags & SNN_F_STATS) != 0;
    c->N = (uint32_t)N;
    c->Np = (uint32_t)std::max<uint64_t>(Np, kPad);
    c->D = cfg->delay + (c->stdp ? 1 : 0);
    c->g_off.assign(cfg->n_inst + 1, 0);
    c->pbase.assign(cfg->n_inst + 1, 0);
    for (uint32_t b = 0; b < cfg->n_inst; ++b) {
        c->g_off[b + 1] = c->g_off[b] + params[b].n;
        c->pbase[b + 1] = c->pbase[b] + (params[b].n + kPad - 1) / kPad * kPad;
    }
    int prio_low = 0, prio_high = 0;
    if (cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high) != cudaSuccess) {
        cudaGetLastError();
        prio_high = 0;
    }
    c->plan_priority = prio_high;
    if (cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
        if (c->side) cudaStreamDestroy(c->side);
        if (c->ev_fork) cudaEventDestroy(c->ev_fork);
        if (c->ev_join) cudaEventDestroy(c->ev_join);
        delete c;
        return SNN_E_CUDA;
    }

    // per-instance constants and Poisson tables
    std::vector<InstDev> hinst(cfg->n_inst);
    // thresholds padded with 0xffffffff: the device sampler searches all 64
    std::vector<uint32_t> hpois((size_t)cfg->n_inst * kPoissonCap, 0xffffffffu);
    for (uint32_t b = 0; b < cfg->n_inst; ++b) {
        int np = 0;
        if (cfg->model != SNN_VOGELS_CUBA) np = poisson_table(params[b].lambda, &hpois[(size_t)b * kPoissonCap], kPoissonCap);
        hinst[b] = make_inst(params[b], c->pbase[b], c->g_off[b], b * kPoissonCap, np);
    }
    // the raster log is shared out in proportion to the instances' neurons
    c->log_lo.assign(cfg->n_inst, 0);
    c->log_n.assign(cfg->n_inst, 0);
    {
        unsigned long long lo = 0;
        const unsigned long long N = c->g_off[cfg->n_inst];
        for (uint32_t b = 0; b < cfg->n_inst; ++b) {
            const unsigned long long share =
                N ? (unsigned long long)((unsigned __int128)cfg->log_capacity * params[b].n / N) : 0ull;
            c->log_lo[b] = hinst[b].log_lo = lo;
            c->log_n[b] = hinst[b].log_n = share;
            lo += share;
        }
    }
    // bucket table of every instance: thresholds below each 2^24 boundary
    std::vector<uint8_t> hstart((size_t)cfg->n_inst * kPoissonBuckets, 0);
    for (uint32_t b = 0; b < cfg->n_inst; ++b) {
        const uint32_t* T = &hpois[(size_t)b * kPoissonCap];
        const uint32_t nT = hinst[b].pois_n;
        uint32_t k = 0;
        for (uint32_t h = 0; h < (uint32_t)kPoissonBuckets; ++h) {
            const uint64_t lo = (uint64_t)h << 24;
            while (k < nT && T[k] < lo) ++k;
            hstart[(size_t)b * kPoissonBuckets + h] = (uint8_t)k;
        }
    }
    std::vector<uint32_t> hmap(c->Np / 32, 0);
    std::vector<uint4> hdesc(c->Np / 32);
    for (uint32_t b = 0; b < cfg->n_inst; ++b)
        for (uint32_t w = c->pbase[b] / 32; w < c->pbase[b + 1] / 32; ++w) {
            hmap[w] = b;
            hdesc[w] = make_uint4(b, c->pbase[b], params[b].n, 0u);
        }

    const size_t Npz = c->Np;
    Net& n = c->net;
    n.Np = c->Np;
    n.D = c->D;
    n.d = cfg->delay;
    n.key0 = cfg->inst_key0;
    n.n_inst = cfg->n_inst;
    n.seed = cfg->seed;
    c->cr = 4;
    while (c->cr < c->D + 2) c->cr <<= 1;
    n.cr = c->cr;
    n.icount = alloc_n<unsigned int>(c, (size_t)c->cr * cfg->n_inst);
    n.ilog = alloc_n<unsigned long long>(c, 2 * (size_t)cfg->n_inst);
    n.inst_spikes = alloc_n<unsigned long long>(c, cfg->n_inst);
    n.tile_ctr = alloc_n<unsigned int>(c, 2);
    c->ctl = alloc_n<Ctl>(c, 1);
    c->inst = alloc_n<InstDev>(c, cfg->n_inst);
    c->inst_of_w32 = alloc_n<uint32_t>(c, Npz / 32);
    c->wdesc = alloc_n<uint4>(c, Npz / 32);
    c->pois = alloc_n<uint32_t>(c, hpois.size());
    c->pois_start = alloc_n<uint8_t>(c, hstart.size());
    n.V = alloc_n<float>(c, Npz);
    n.r = alloc_n<uint8_t>(c, Npz);
    n.acc0 = alloc_n<int32_t>(c, Npz);
    n.q = alloc_n<uint32_t>(c, (size_t)c->D * Npz);
    bool ok = c->ctl && c->inst && c->inst_of_w32 && c->wdesc && c->pois && c->pois_start && n.V && n.r && n.acc0 && n.q && n.icount && n.ilog &&
              n.inst_spikes && n.tile_ctr;
    if (c->generic) {
        c->mstate = dev_alloc(c, c->mbytes * Npz);
        ok = ok && c->mstate;
    }
    if (c->vogels) {
        n.ge = alloc_n<float>(c, Npz);
        n.gi = alloc_n<float>(c, Npz);
        n.acc1 = alloc_n<int32_t>(c, Npz);
        ok = ok && n.ge && n.gi && n.acc1;
    }
    if (c->stdp) {
        n.x = alloc_n<float>(c, Npz);
        n.y = alloc_n<float>(c, Npz);
        n.bits = alloc_n<uint32_t>(c, (size_t)c->D * (Npz / 32));
        ok = ok && n.x && n.y && n.bits;
    }
    if (c->lazy) {
        n.F = cfg->lazy_fifo ? cfg->lazy_fifo : (uint32_t)kLazyMaxF;
        n.hist = alloc_n<unsigned long long>(c, 2 * Npz);
        n.yring = alloc_n<float>(c, (size_t)n.F * Npz);
        n.age = alloc_n<uint32_t>(c, Npz);
        n.xq = alloc_n<uint32_t>(c, Npz);
        n.xcount = alloc_n<unsigned int>(c, 2);
        ok = ok && n.hist && n.yring && n.age && n.xq && n.xcount;
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stdp_lazy<true>, kLazyThreads, 0) != cudaSuccess)
            cudaGetLastError();
        c->lazy_blocks = (uint32_t)sm_count() * (uint32_t)std::max(1, per_sm);
    }
    if (c->stats) {
        n.st_cnt = alloc_n<uint32_t>(c, Npz);
        n.st_last = alloc_n<uint32_t>(c, Npz);
        n.st_sum = alloc_n<unsigned long long>(c, Npz);
        n.st_sq = alloc_n<unsigned long long>(c, Npz);
        ok = ok && n.st_cnt && n.st_last && n.st_sum && n.st_sq;
    }
    if (cfg->log_capacity) {
        n.log = alloc_n<unsigned long long>(c, cfg->log_capacity);
        n.log_cap = cfg->log_capacity;
        ok = ok && n.log;
    }
    if (!ok) {
        snn_destroy(c);
        return SNN_E_NOMEM;
    }
    n.ctl = c->ctl;
    n.inst = c->inst;
    n.inst_of_w32 = c->inst_of_w32;
    n.wdesc = c->wdesc;
    n.pois = c->pois;
    n.pois_start = c->pois_start;
    cudaError_t e = cudaMemcpyAsync(c->inst, hinst.data(), hinst.size() * sizeof(InstDev), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->inst_of_w32, hmap.data(), hmap.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->wdesc, hdesc.data(), hdesc.size() * sizeof(uint4), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pois, hpois.data(), hpois.size() * 4, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(c->pois_start, hstart.data(), hstart.size(), cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->ctl, 0, sizeof(Ctl), c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        snn_destroy(c);
        return SNN_E_CUDA;
    }
    *out = c;
    return SNN_OK;
}

// The STDP column index (coff, cedge, cpre) of the loaded graph: k_col_count,
// an exclusive scan, k_col_fill.  Needs the mapped targets and meta.
snn_status build_columns(snn_ctx* c)
{
    const uint32_t Np = c->Np;
    cudaStream_t s = c->stream;
    Net n = c->net;
    n.roff = c->roff;
    n.tgt = c->tgt;
    n.meta = c->meta;
    unsigned long long* cnt = alloc_n<unsigned long long>(c, (size_t)Np + 1);
    unsigned long long* cur = alloc_n<unsigned long long>(c, (size_t)Np + 1);
    c->coff = alloc_n<uint64_t>(c, (size_t)Np + 1);
    void* tmp = nullptr;
    auto done = [&](snn_status st) {
        dev_free(c, cnt);
        dev_free(c, cur);
        dev_free(c, tmp);
        return st;
    };
    if (!cnt || !cur || !c->coff) return done(fail(c, SNN_E_NOMEM, "STDP column index allocation failed"));
    const uint32_t grid = (uint32_t)sm_count() * 16;
    size_t tmp_bytes = 0;
    cudaError_t e = cudaMemsetAsync(cnt, 0, ((size_t)Np + 1) * 8, s);
    if (e == cudaSuccess) {
        k_col_count<<<grid, 256, 0, s>>>(n, cnt);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(nullptr, tmp_bytes, cnt, cur, (int64_t)Np + 1, s);
    if (e == cudaSuccess && !(tmp = dev_alloc(c, std::max<size_t>(tmp_bytes, 16)))) e = cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, cnt, cur, (int64_t)Np + 1, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(c->coff, cur, ((size_t)Np + 1) * 8, cudaMemcpyDeviceToDevice, s);
    unsigned long long P = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&P, cur + Np, 8, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fail(c, SNN_E_CUDA, "STDP column index: %s", cudaGetErrorString(e)));
    c->cedge = alloc_n<uint32_t>(c, P ? P : 1);
    c->cpre = alloc_n<uint32_t>(c, P ? P : 1);
    if (!c->cedge || !c->cpre) return done(fail(c, SNN_E_NOMEM, "STDP column index allocation failed"));
    k_col_fill<<<grid, 256, 0, s>>>(n, cur, c->cedge, c->cpre);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return done(fail(c, SNN_E_CUDA, "STDP column index: %s", cudaGetErrorString(e)));
    return done(SNN_OK);
}

// snn_build_graph with one weight per edge (w_q) or per row (w_row).
snn_status build_graph(snn_ctx* c, const uint64_t* row_off, const uint32_t* tgt_h, const int32_t* w_q,
                       const int32_t* w_row)
{
    if (!c) return SNN_E_ARG;
    if (!row_off) return fail(c, SNN_E_ARG, "row_off is NULL");
    const uint32_t N = c->N;
    if (row_off[0] != 0) return fail(c, SNN_E_ARG, "row_off[0] must be 0");
    for (uint32_t j = 0; j < N; ++j)
        if (row_off[j + 1] < row_off[j]) return fail(c, SNN_E_ARG, "row_off decreases at row %u", j);
    const uint64_t E = row_off[N];
    if (E && (!tgt_h || (!w_q && !w_row))) return fail(c, SNN_E_ARG, "tgt/w_q is NULL");
    if (c->stdp && E >= (1ull << 32)) return fail(c, SNN_E_ARG, "STDP needs fewer than 2^32 edges");

    // drop a previous graph
    drop_graphs(c);
    tiled_free(c->tiled, [c](void* p) { dev_free(c, p); });
    c->use_tiled = false;
    for (void* p : {(void*)c->roff, (void*)c->tgt, (void*)c->w16p, (void*)c->w32p, (void*)c->meta, (void*)c->coff,
                    (void*)c->cedge, (void*)c->cpre, (void*)c->w_init, (void*)c->rinfo, (void*)c->pk32})
        dev_free(c, p);
    dev_free(c, c->roww);
    c->roww = nullptr;
    c->net.roww = nullptr;
    c->rinfo = nullptr;
    c->pk32 = nullptr;
    c->packed = false;
    c->net.pk = nullptr;
    dev_free(c, c->pk16);
    c->pk16 = nullptr;
    c->off16 = false;
    c->net.pk16 = nullptr;
    c->roff = nullptr; c->tgt = nullptr; c->w16p = nullptr; c->w32p = nullptr; c->meta = nullptr;
    c->coff = nullptr; c->cedge = nullptr; c->cpre = nullptr; c->w_init = nullptr;
    c->graph_loaded = false;

    // padded row offsets and the row -> (source, instance) maps
    const uint32_t Np = c->Np;
    std::vector<uint64_t> hroff((size_t)Np + 1, 0);
    std::vector<uint32_t> hsrc((size_t)Np, 0xffffffffu), hinst((size_t)Np, 0);
    {
        uint32_t b = 0;
        for (uint32_t pj = 0; pj < Np; ++pj) {
            while (b + 1 < c->cfg.n_inst && pj >= c->pbase[b + 1]) ++b;
            hinst[pj] = b;
            const uint32_t local = pj - c->pbase[b];
            if (pj < c->pbase[b + 1] && local < c->params[b].n) {
                const uint32_t j = c->g_off[b] + local;
                hsrc[pj] = j;
                hroff[pj] = row_off[j];
            } else {
                // padding: an empty row at the offset of the next real row
                const uint32_t next_g = c->g_off[b] + std::min(local, c->params[b].n);
                hroff[pj] = row_off[std::min(next_g, N)];
            }
        }
        hroff[Np] = E;
        for (uint32_t pj = Np; pj-- > 0;)
            if (hsrc[pj] == 0xffffffffu) hroff[pj] = hroff[pj + 1];
    }

    c->E = E;
    c->roff = alloc_n<uint64_t>(c, (size_t)Np + 1);
    c->tgt = alloc_n<uint32_t>(c, E + 16);  // tail padding: bulk copies round their end up
    c->meta = alloc_n<uint8_t>(c, Np);
    if (c->w16)
        c->w16p = alloc_n<int16_t>(c, E + 16);
    else
        c->w32p = alloc_n<float>(c, E + 16);
    if (c->stdp) c->w_init = alloc_n<int32_t>(c, E);
    int32_t* wtmp = c->stdp ? c->w_init : alloc_n<int32_t>(c, E);
    uint32_t* dsrc = alloc_n<uint32_t>(c, Np);
    uint32_t* dinst = alloc_n<uint32_t>(c, Np);
    uint32_t* dgoff = alloc_n<uint32_t>(c, c->cfg.n_inst + 1);
    uint32_t* dpb = alloc_n<uint32_t>(c, c->cfg.n_inst + 1);
    uint32_t* dnexc = alloc_n<uint32_t>(c, c->cfg.n_inst);
    unsigned int* dunsorted = alloc_n<unsigned int>(c, 1);
    auto cleanup_tmp = [&]() {
        if (!c->stdp) dev_free(c, wtmp);
        dev_free(c, dsrc); dev_free(c, dinst); dev_free(c, dgoff); dev_free(c, dpb); dev_free(c, dnexc);
        dev_free(c, dunsorted);
    };
    if (!c->roff || !c->tgt || !c->meta || (c->w16 ? !c->w16p : !c->w32p) || !wtmp || !dsrc || !dinst || !dgoff ||
        !dpb || !dnexc || !dunsorted) {
        cleanup_tmp();
        return fail(c, SNN_E_NOMEM, "device allocation for a graph of %llu edges failed", (unsigned long long)E);
    }
    std::vector<uint32_t> hnexc(c->cfg.n_inst);
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b) hnexc[b] = c->params[b].n_exc;
    cudaStream_t s = c->stream;
    CUDA_TRY(c, cudaMemcpyAsync(c->roff, hroff.data(), hroff.size() * 8, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(dsrc, hsrc.data(), hsrc.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(dinst, hinst.data(), hinst.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(dgoff, c->g_off.data(), c->g_off.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(dpb, c->pbase.data(), c->pbase.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(c, cudaMemcpyAsync(dnexc, hnexc.data(), hnexc.size() * 4, cudaMemcpyHostToDevice, s));
    if (E) {
        snn_status up = upload(c, c->tgt, tgt_h, E * 4, s);
        if (up == SNN_OK && w_q) up = upload(c, wtmp, w_q, E * 4, s);
        if (up == SNN_OK && !w_q) {  // one weight per row: spread over the row's edges on the device
            int32_t* dwr = alloc_n<int32_t>(c, N);
            if (!dwr) {
                up = fail(c, SNN_E_NOMEM, "row weights");
            } else {
                up = upload(c, dwr, w_row, (size_t)N * 4, s);
                if (up == SNN_OK) {
                    k_spread_row_weights<<<(uint32_t)sm_count() * 16, 256, 0, s>>>(c->roff, dsrc, dwr, Np, wtmp);
                    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
                        up = fail(c, SNN_E_CUDA, "row weights");
                }
                dev_free(c, dwr);
            }
        }
        if (up != SNN_OK) {
            cleanup_tmp();
            return up;
        }
    }
    CUDA_TRY(c, cudaMemsetAsync(&c->ctl->err, 0, sizeof(unsigned int), s));
    CUDA_TRY(c, cudaMemsetAsync(dunsorted, 0, sizeof(unsigned int), s));
    RowMapArgs a{};
    a.roff = c->roff; a.row_src = dsrc; a.row_inst = dinst; a.g_inst_off = dgoff; a.pbase = dpb; a.n_exc = dnexc;
    a.tgt = c->tgt; a.wq = wtmp; a.w16 = c->w16p; a.w32 = c->w32p; a.meta = c->meta; a.Np = Np;
    a.w16_mode = c->w16 ? 1 : 0; a.vogels = c->vogels ? 1 : 0; a.stdp = c->stdp ? 1 : 0; a.err = &c->ctl->err;
    a.unsorted = dunsorted;
    k_map_rows<<<(uint32_t)sm_count() * 16, 256, 0, s>>>(a);
    CUDA_TRY(c, cudaGetLastError());
    unsigned int err = 0, unsorted = 0;
    CUDA_TRY(c, cudaMemcpyAsync(&err, &c->ctl->err, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaMemcpyAsync(&unsorted, dunsorted, 4, cudaMemcpyDeviceToHost, s));
    CUDA_TRY(c, cudaStreamSynchronize(s));
    cleanup_tmp();
    c->rows_sorted = unsorted == 0;
    if (err) {
        if (err & kErrBadTarget) return fail(c, SNN_E_ARG, "a row has a target outside its source's instance");
        if (err & kErrPlasticShift)
            return fail(c, SNN_E_ARG, "plastic (excitatory) rows need weights within int16 lattice units");
        return fail(c, SNN_E_ARG, c->w16 ? "a row's weights are not int16 codes times one power of two"
                                         : "a weight exceeds 2^24 lattice units");
    }

    // STDP column index: plastic in-edges (exc -> exc) of every padded post id
    // (eager potentiation only; the lazy replay walks rows), built on the device
    if (c->stdp && !c->lazy) {
        snn_status cs = build_columns(c);
        if (cs != SNN_OK) return cs;
    }

    c->rinfo = alloc_n<uint4>(c, Np);
    if (!c->rinfo) return fail(c, SNN_E_NOMEM, "row records");
    k_row_info<<<(uint32_t)sm_count() * 8, 256, 0, s>>>(c->roff, c->meta, Np, c->rinfo);
    CUDA_TRY(c, cudaGetLastError());

    Net& n = c->net;
    n.rinfo = c->rinfo;
    n.roff = c->roff;
    n.meta = c->meta;
    n.w16 = c->w16p;
    {
        bool changed = false;
        snn_status st = refresh_row_weights(c, &changed);
        if (st != SNN_OK) return st;
    }
    n.roff = c->roff;
    n.tgt = c->tgt;
    n.w16 = c->w16p;
    n.w32 = c->w32p;
    n.meta = c->meta;
    n.coff = c->coff;
    n.cedge = c->cedge;
    n.cpre = c->cpre;

    // receive strategy: the target-tiled form needs sorted rows
    c->inst_edges.assign(c->cfg.n_inst, 0);
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b)
        c->inst_edges[b] = row_off[c->g_off[b + 1]] - row_off[c->g_off[b]];
    c->use_tiled = false;
    c->use_bulk = false;
    c->tune_count = 0;
    c->tune_next = c->cfg.tune_steps ? c->cfg.tune_steps : 256;
    c->spk_seen.assign(c->cfg.n_inst, 0);
    {
        // row records hold a row's length in 32 bits
        uint64_t max_deg = 0;
        for (uint32_t j = 0; j < N; ++j) max_deg = std::max<uint64_t>(max_deg, row_off[j + 1] - row_off[j]);
        c->tiled_fits = max_deg < (1ull << 32);
    }
    c->k_steps = c->cfg.steps_per_graph ? c->cfg.steps_per_graph : 16;
    c->tuned = false;
    for (float& x : c->tune_ms) x = 0.f;
    c->graph_loaded = true;
    snn_status st = SNN_OK;
    if (c->cfg.receive == SNN_RECV_AUTO) {
        st = tune_receive(c);
        c->tuned = st == SNN_OK;
    } else if (c->cfg.receive == SNN_RECV_GLOBAL) {
        st = use_form(c, kFormGlobal);
    } else if (c->cfg.receive == SNN_RECV_PERSISTENT) {
        st = persist_applies(c) ? use_form(c, kFormPersist) : fail(c, SNN_E_ARG, "the persistent launch needs a fixed model without plasticity");
    } else if (!c->rows_sorted || !c->tiled_fits) {
        st = fail(c, SNN_E_ARG, c->rows_sorted ? "the tiled receive does not fit this graph"
                                               : "the tiled receive needs rows sorted by target");
    } else if (c->cfg.receive == SNN_RECV_BULK) {
        st = use_form(c, kFormBulk);
    } else {
        c->use_tiled = true;
        c->use_bulk = false;
        const bool fuse = fused_applies(c) && !(c->cfg.flags & SNN_F_SERIAL);
        st = use_form(c, fuse ? kFormFused : kFormTiled);
        if (st == SNN_E_ARG && fuse) st = use_form(c, kFormTiled);  // the fused kernel did not fit
    }
    if (st != SNN_OK) {
        c->graph_loaded = false;
        return st;
    }
    st = reset_state(c);
    if (st != SNN_OK) return st;
    CUDA_TRY(c, cudaStreamSynchronize(s));
    return SNN_OK;
}

snn_status snn_build_graph(snn_ctx* c, const uint64_t* row_off, const uint32_t* tgt, const int32_t* w_q)
{
    return build_graph(c, row_off, tgt, w_q, nullptr);
}

snn_status snn_build_graph_rows(snn_ctx* c, const uint64_t* row_off, const uint32_t* tgt, const int32_t* w_row)
{
    if (c && c->N && !w_row) return fail(c, SNN_E_ARG, "w_row is NULL");
    return build_graph(c, row_off, tgt, nullptr, w_row);
}

snn_status snn_reset(snn_ctx* c)
{
    if (!c) return SNN_E_ARG;
    if (!c->graph_loaded) return fail(c, SNN_E_STATE, "no graph loaded");
    snn_status st = reset_state(c);
    if (st != SNN_OK) return st;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    return SNN_OK;
}

snn_status snn_step(snn_ctx* c, uint32_t n_steps)
{
    if (!c) return SNN_E_ARG;
    if (!c->graph_loaded) return fail(c, SNN_E_STATE, "snn_step before snn_build_graph");
    uint32_t left = n_steps;
    // re-plan the static plan of the bulk-copy receive twice, at tune_steps
    // and 8 x tune_steps (the tiled receive plans every step on the device)
    while (c->use_tiled && c->use_bulk && c->tune_count < 2 && c->cfg.tune_steps != 0xffffffffu &&
           c->host_steps + left >= c->tune_next) {
        uint32_t first = (uint32_t)(c->tune_next > c->host_steps ? c->tune_next - c->host_steps : 0);
        left -= first;
        c->host_steps += first;
        while (c->gk && first >= c->k_steps) {
            CUDA_TRY(c, cudaGraphLaunch(c->gk, c->stream));
            first -= c->k_steps;
        }
        while (first--) CUDA_TRY(c, cudaGraphLaunch(c->g1, c->stream));
        snn_status st = retune(c);
        if (st != SNN_OK) return st;
        c->tune_next *= 8;
    }
    c->host_steps += left;
    return run_steps(c, left);
}

snn_status snn_step_profiled(snn_ctx* c, uint32_t n_steps, double* phase_ms)
{
    if (!c || !phase_ms) return SNN_E_ARG;
    if (!c->graph_loaded) return fail(c, SNN_E_STATE, "snn_step_profiled before snn_build_graph");
    for (int k = 0; k < kPhases; ++k) phase_ms[k] = 0.0;
    std::vector<cudaEvent_t> ev((size_t)n_steps * (kPhases + 1));
    for (auto& e : ev)
        if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        }
    snn_status st = SNN_OK;
    for (uint32_t i = 0; i < n_steps && st == SNN_OK; ++i) {
        for (int k = 0; k <= kPhases; ++k)
            if (!ev[(size_t)i * (kPhases + 1) + k]) st = fail(c, SNN_E_CUDA, "cudaEventCreate failed");
        if (st != SNN_OK) break;
        cudaEvent_t* e = &ev[(size_t)i * (kPhases + 1)];
        if (c->persistent) {  // the whole step is one launch: phase [3]
            for (int k = 0; k <= 3; ++k) cudaEventRecord(e[k], c->stream);
            st = launch_persistent(c, 1);
            for (int k = 4; k <= kPhases; ++k) cudaEventRecord(e[k], c->stream);
        } else {
            st = enqueue_step(c, c->stream, e);
        }
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (st == SNN_OK && e != cudaSuccess) st = fail(c, SNN_E_CUDA, "profiled steps: %s", cudaGetErrorString(e));
    for (uint32_t i = 0; i < n_steps && st == SNN_OK; ++i)
        for (int k = 0; k < kPhases; ++k) {
            float ms = 0.f;
            const size_t b = (size_t)i * (kPhases + 1) + k;
            if (cudaEventElapsedTime(&ms, ev[b], ev[b + 1]) == cudaSuccess)
                phase_ms[k] += ms;
        }
    for (auto& x : ev)
        if (x) cudaEventDestroy(x);
    c->host_steps += n_steps;
    return st;
}

snn_status snn_sync(snn_ctx* c)
{
    if (!c) return SNN_E_ARG;
    return check_device_errors(c);
}

snn_status snn_read_spikes(snn_ctx* c, uint32_t t0, uint32_t t1, uint32_t* steps, uint32_t* ids, uint64_t cap,
                           uint64_t* n_out)
{
    if (!c || !n_out) return SNN_E_ARG;
    *n_out = 0;
    if (!c->cfg.log_capacity) return fail(c, SNN_E_STATE, "the context has no spike log (log_capacity = 0)");
    if (cap && (!steps || !ids)) return fail(c, SNN_E_ARG, "NULL output with cap > 0");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    Ctl h;
    CUDA_TRY(c, cudaMemcpy(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost));
    // logged spikes of each instance: its count before the last step plus the
    // last step's queue index (the next step's update would compute the same)
    const uint32_t B = c->cfg.n_inst;
    std::vector<unsigned long long> avail(B, 0);
    bool overflow = false;
    if (h.t > h.t_log0) {
        std::vector<unsigned int> ic(B, 0);
        CUDA_TRY(c, cudaMemcpy(avail.data(), c->net.ilog + (size_t)((h.t - 1) & 1ull) * B, B * 8, cudaMemcpyDeviceToHost));
        CUDA_TRY(c, cudaMemcpy(ic.data(), c->net.icount + (size_t)((h.t - 1) & (c->cr - 1)) * B, B * 4,
                               cudaMemcpyDeviceToHost));
        for (uint32_t b = 0; b < B; ++b) {
            avail[b] += ic[b];
            overflow = overflow || avail[b] > c->log_n[b];
            avail[b] = std::min<unsigned long long>(avail[b], c->log_n[b]);
        }
    }
    // each region is in step order (steps append after the previous ones), so
    // the entries of steps [t0, t1) are one range of it, found by bisection
    std::vector<unsigned long long> rng(2 * (size_t)B, 0);
    {
        unsigned long long* d_av = alloc_n<unsigned long long>(c, B);
        unsigned long long* d_rg = alloc_n<unsigned long long>(c, 2 * (size_t)B);
        cudaError_t e = (d_av && d_rg) ? cudaSuccess : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_av, avail.data(), B * 8, cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess) {
            k_log_ranges<<<grid_for(B, 128), 128, 0, c->stream>>>(c->net, d_av, t0, t1, d_rg);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(rng.data(), d_rg, rng.size() * 8, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, d_av);
        dev_free(c, d_rg);
        if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "raster ranges: %s", cudaGetErrorString(e));
    }
    uint64_t n = 0;
    for (uint32_t b = 0; b < B; ++b) n += rng[2 * b + 1] - rng[2 * b];
    *n_out = n;
    if (overflow)
        return fail(c, SNN_E_OVERFLOW, "the spike log overflowed (an instance filled its share; capacity %llu)",
                    (unsigned long long)c->cfg.log_capacity);
    if (cap == 0 || n == 0) return SNN_OK;
    if (cap < n) return fail(c, SNN_E_OVERFLOW, "output capacity %llu < %llu spikes", (unsigned long long)cap,
                            (unsigned long long)n);
    // the ranges in chunks of at most 4,096 entries, one block each
    std::vector<LogChunk> hc;
    {
        unsigned long long dst = 0;
        for (uint32_t b = 0; b < B; ++b)
            for (unsigned long long i = rng[2 * b]; i < rng[2 * b + 1]; i += 4096) {
                const unsigned long long len = std::min<unsigned long long>(4096, rng[2 * b + 1] - i);
                hc.push_back(LogChunk{c->log_lo[b] + i, dst, (uint32_t)len, b});
                dst += len;
            }
    }
    // keys (step - t0) << 32 | global id, radix-sorted on the device, split
    // into the two output arrays
    const uint64_t t_hi = std::min<uint64_t>(t1, h.t);
    int end_bit = 32;
    while (end_bit < 64 && (t_hi - t0) >= (1ull << (end_bit - 32))) ++end_bit;
    unsigned long long* ka = alloc_n<unsigned long long>(c, n);
    unsigned long long* kb = alloc_n<unsigned long long>(c, n);
    size_t tmp_bytes = 0;
    cub::DoubleBuffer<unsigned long long> db(ka, kb);
    void* tmp = nullptr;
    cudaError_t e = cudaSuccess;
    if (ka && kb) {
        LogChunk* d_ch = alloc_n<LogChunk>(c, hc.size());
        e = d_ch ? cudaMemcpyAsync(d_ch, hc.data(), hc.size() * sizeof(LogChunk), cudaMemcpyHostToDevice, c->stream)
                 : cudaErrorMemoryAllocation;
        if (e == cudaSuccess) {
            k_raster_keys<<<(uint32_t)hc.size(), 256, 0, c->stream>>>(c->net, d_ch, t0, ka);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);  // the chunk list is freed next
        dev_free(c, d_ch);
        if (e == cudaSuccess) e = cub::DeviceRadixSort::SortKeys(nullptr, tmp_bytes, db, (int64_t)n, 0, end_bit, c->stream);
        if (e == cudaSuccess) tmp = dev_alloc(c, std::max<size_t>(tmp_bytes, 16));
    }
    if (!ka || !kb || !tmp) {
        dev_free(c, ka);
        dev_free(c, kb);
        dev_free(c, tmp);
        return fail(c, e == cudaSuccess ? SNN_E_NOMEM : SNN_E_CUDA, "raster sort buffers");
    }
    e = cub::DeviceRadixSort::SortKeys(tmp, tmp_bytes, db, (int64_t)n, 0, end_bit, c->stream);
    uint32_t* split = reinterpret_cast<uint32_t*>(db.Alternate());  // steps then ids, n each
    if (e == cudaSuccess) {
        k_raster_split<<<grid_for(n, 256), 256, 0, c->stream>>>(db.Current(), n, t0, split, split + n);
        e = cudaGetLastError();
    }
    snn_status out = SNN_OK;
    if (e == cudaSuccess) out = download(c, steps, split, n * 4, c->stream);
    if (e == cudaSuccess && out == SNN_OK) out = download(c, ids, split + n, n * 4, c->stream);
    dev_free(c, tmp);
    dev_free(c, ka);
    dev_free(c, kb);
    if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "raster readout: %s", cudaGetErrorString(e));
    return out;
}

snn_status snn_log_clear(snn_ctx* c)
{
    if (!c) return SNN_E_ARG;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    Ctl* d = c->ctl;
    unsigned long long t = 0;
    CUDA_TRY(c, cudaMemcpy(&t, &d->t, 8, cudaMemcpyDeviceToHost));
    unsigned int err = 0;
    CUDA_TRY(c, cudaMemcpy(&d->t_log0, &t, 8, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemcpy(&err, &d->err, 4, cudaMemcpyDeviceToHost));
    err &= ~kErrLogOverflow;
    CUDA_TRY(c, cudaMemcpy(&d->err, &err, 4, cudaMemcpyHostToDevice));
    return SNN_OK;
}

static snn_status field_ptr(snn_ctx* c, snn_field f, void** p, size_t* elem, bool* u8)
{
    *u8 = false;
    *elem = 4;
    switch (f) {
    case SNN_FIELD_V: *p = c->net.V; break;
    case SNN_FIELD_GE: *p = c->net.ge; break;
    case SNN_FIELD_GI: *p = c->net.gi; break;
    case SNN_FIELD_R: *p = c->net.r; *u8 = true; break;
    case SNN_FIELD_X: *p = c->net.x; break;
    case SNN_FIELD_Y: *p = c->net.y; break;
    case SNN_FIELD_ACC0: {  // the input of the next update: with the fused step, buffer t & 1
        *p = c->net.acc0;
        if (c->fused) {
            unsigned long long t = 0;
            CUDA_TRY(c, cudaMemcpy(&t, &c->ctl->t, 8, cudaMemcpyDeviceToHost));
            if (t & 1ull) *p = c->net.accx;
        }
        break;
    }
    case SNN_FIELD_ACC1: *p = c->net.acc1; break;
    case SNN_FIELD_MODEL: *p = c->mstate; *elem = c->mbytes; break;
    default: return fail(c, SNN_E_ARG, "unknown field %d", (int)f);
    }
    if (!*p) return fail(c, SNN_E_ARG, "field %d does not exist for this model", (int)f);
    return SNN_OK;
}

snn_status snn_read_state(snn_ctx* c, snn_field f, void* host)
{
    if (!c || !host) return SNN_E_ARG;
    if (!c->graph_loaded) return fail(c, SNN_E_STATE, "no graph loaded");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (f == SNN_FIELD_W || f == SNN_FIELD_X) {
        snn_status st = lazy_flush(c);
        if (st != SNN_OK) return st;
    }
    if (f == SNN_FIELD_W) {
        int32_t* tmp = alloc_n<int32_t>(c, c->E);
        if (!tmp) return fail(c, SNN_E_NOMEM, "temporary weight buffer");
        k_weights_out<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->roff, c->meta, c->w16p, c->w32p,
                                                                         c->w16 ? 1 : 0, c->Np, tmp);
        cudaError_t e = cudaGetLastError();
        if (e == cudaSuccess && c->E) e = cudaMemcpyAsync(host, tmp, c->E * 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, tmp);
        if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "weight readback: %s", cudaGetErrorString(e));
        return SNN_OK;
    }
    void* p;
    size_t elem;
    bool u8;
    snn_status st = field_ptr(c, f, &p, &elem, &u8);
    if (st != SNN_OK) return st;
    const size_t esz = u8 ? 1 : elem;
    std::vector<uint8_t> buf((size_t)c->Np * esz);
    CUDA_TRY(c, cudaMemcpy(buf.data(), p, buf.size(), cudaMemcpyDeviceToHost));
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b)
        for (uint32_t l = 0; l < c->params[b].n; ++l) {
            const uint32_t pid = c->pbase[b] + l, g = c->g_off[b] + l;
            if (u8)
                static_cast<int32_t*>(host)[g] = buf[pid];
            else
                std::memcpy(static_cast<uint8_t*>(host) + (size_t)g * esz, buf.data() + (size_t)pid * esz, esz);
        }
    return SNN_OK;
}

snn_status snn_write_state(snn_ctx* c, snn_field f, const void* host)
{
    if (!c || !host) return SNN_E_ARG;
    if (!c->graph_loaded) return fail(c, SNN_E_STATE, "no graph loaded");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    if (f == SNN_FIELD_W || f == SNN_FIELD_X) {
        snn_status st = lazy_flush(c);
        if (st != SNN_OK) return st;
    }
    if (f == SNN_FIELD_W) {
        int32_t* tmp = alloc_n<int32_t>(c, c->E);
        if (!tmp) return fail(c, SNN_E_NOMEM, "temporary weight buffer");
        unsigned int err = 0;
        cudaError_t e = c->E ? cudaMemcpyAsync(tmp, host, c->E * 4, cudaMemcpyHostToDevice, c->stream) : cudaSuccess;
        if (e == cudaSuccess) e = cudaMemsetAsync(&c->ctl->err, 0, 4, c->stream);
        if (e == cudaSuccess) {
            k_weights_in<<<(uint32_t)sm_count() * 16, 256, 0, c->stream>>>(c->roff, c->meta, tmp, c->w16 ? 1 : 0,
                                                                            c->Np, c->w16p, c->w32p, &c->ctl->err);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &c->ctl->err, 4, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        dev_free(c, tmp);
        if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "weight upload: %s", cudaGetErrorString(e));
        if (err & kErrBadWeight) return fail(c, SNN_E_ARG, "a weight does not fit its row's int16 code and shift");
        snn_status st = pack_edges(c);
        if (st == SNN_OK) CUDA_TRY(c, cudaStreamSynchronize(c->stream));
        bool changed = false;
        if (st == SNN_OK) st = refresh_row_weights(c, &changed);
        if (st == SNN_OK && changed) st = use_form(c, c->form);  // the receive reads another layout now
        return st;
    }
    void* p;
    size_t elem;
    bool u8;
    snn_status st = field_ptr(c, f, &p, &elem, &u8);
    if (st != SNN_OK) return st;
    const size_t esz = u8 ? 1 : elem;
    std::vector<uint8_t> buf((size_t)c->Np * esz);
    CUDA_TRY(c, cudaMemcpy(buf.data(), p, buf.size(), cudaMemcpyDeviceToHost));
    for (uint32_t b = 0; b < c->cfg.n_inst; ++b)
        for (uint32_t l = 0; l < c->params[b].n; ++l) {
            const uint32_t pid = c->pbase[b] + l, g = c->g_off[b] + l;
            if (u8) {
                const int32_t v = static_cast<const int32_t*>(host)[g];
                if (v < 0 || v > 255) return fail(c, SNN_E_ARG, "refractory count out of range");
                buf[pid] = (uint8_t)v;
            } else {
                std::memcpy(buf.data() + (size_t)pid * esz, static_cast<const uint8_t*>(host) + (size_t)g * esz, esz);
            }
        }
    CUDA_TRY(c, cudaMemcpy(p, buf.data(), buf.size(), cudaMemcpyHostToDevice));
    return SNN_OK;
}

snn_status snn_counters(snn_ctx* c, uint64_t* steps, uint64_t* spikes, uint64_t* events)
{
    if (!c) return SNN_E_ARG;
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    Ctl h;
    CUDA_TRY(c, cudaMemcpy(&h, c->ctl, sizeof h, cudaMemcpyDeviceToHost));
    unsigned long long last = 0;  // the last step's spikes are folded in by the next update
    if (h.t > 0) {
        std::vector<unsigned int> ic(c->cfg.n_inst, 0);
        CUDA_TRY(c, cudaMemcpy(ic.data(), c->net.icount + (size_t)((h.t - 1) & (c->cr - 1)) * c->cfg.n_inst,
                               ic.size() * 4, cudaMemcpyDeviceToHost));
        for (unsigned int x : ic) last += x;
    }
    if (steps) *steps = h.t;
    if (spikes) *spikes = h.spikes + last;
    if (events) *events = h.events;
    return SNN_OK;
}

snn_status snn_stats(snn_ctx* c, uint32_t inst, double* rate_hz, double* isi_cv)
{
    if (!c || inst >= c->cfg.n_inst) return SNN_E_ARG;
    if (!c->stats) return fail(c, SNN_E_STATE, "the context was created without SNN_F_STATS");
    double* d = alloc_n<double>(c, 3);
    if (!d) return fail(c, SNN_E_NOMEM, "stats buffer");
    double h[3] = {0, 0, 0};
    Ctl hc;
    cudaError_t e = cudaMemsetAsync(d, 0, 3 * sizeof(double), c->stream);
    if (e == cudaSuccess) {
        k_stats<<<64, 256, 0, c->stream>>>(c->net.st_cnt, c->net.st_sum, c->net.st_sq, c->pbase[inst],
                                           c->pbase[inst] + c->params[inst].n, d);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, sizeof h, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hc, c->ctl, sizeof hc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    dev_free(c, d);
    if (e != cudaSuccess) return fail(c, SNN_E_CUDA, "stats: %s", cudaGetErrorString(e));
    const double window = (double)(hc.t - hc.t_stat0) * c->params[inst].dt * 1e-3;
    if (rate_hz) *rate_hz = (window > 0 && c->params[inst].n) ? h[0] / c->params[inst].n / window : 0.0;
    if (isi_cv) *isi_cv = h[2] > 0 ? h[1] / h[2] : 0.0;
    return SNN_OK;
}

snn_status snn_stats_clear(snn_ctx* c)
{
    if (!c) return SNN_E_ARG;
    if (!c->stats) return fail(c, SNN_E_STATE, "the context was created without SNN_F_STATS");
    CUDA_TRY(c, cudaStreamSynchronize(c->stream));
    unsigned long long t = 0;
    CUDA_TRY(c, cudaMemcpy(&t, &c->ctl->t, 8, cudaMemcpyDeviceToHost));
    CUDA_TRY(c, cudaMemcpy(&c->ctl->t_stat0, &t, 8, cudaMemcpyHostToDevice));
    CUDA_TRY(c, cudaMemset(c->net.st_cnt, 0, (size_t)c->Np * 4));
    CUDA_TRY(c, cudaMemset(c->net.st_sum, 0, (size_t)c->Np * 8));
    CUDA_TRY(c, cudaMemset(c->net.st_sq, 0, (size_t)c->Np * 8));
    return SNN_OK;
}

snn_status snn_get_info(snn_ctx* c, snn_info* info)
{
    if (!c || !info) return SNN_E_ARG;
    info->receive = c->use_tiled ? (c->use_bulk ? SNN_RECV_BULK : SNN_RECV_TILED) : SNN_RECV_GLOBAL;
    info->n_tiles = c->use_tiled ? c->tiled.n_tiles : 0;
    info->n_padded = c->Np;
    info->rows_sorted = c->rows_sorted ? 1 : 0;
    info->edges = c->E;
    info->device_bytes = c->bytes_held;
    info->edge_bytes = c->use_tiled ? edge_bytes_of(recv_wm(c)) : (c->net.roww ? 4u : (c->w16 ? 6u : 8u));
    info->model_state_bytes = (uint32_t)c->mbytes;
    info->fused = c->fused ? 1u : 0u;
    info->tuned = c->tuned ? 1u : 0u;
    for (int f = 0; f < 5; ++f) info->tune_ms[f] = c->tune_ms[f];
    info->persistent = c->persistent ? 1u : 0u;
    info->persist_ctas = c->persistent ? c->persist_grid : 0u;
    return SNN_OK;
}

void snn_destroy(snn_ctx* c)
{
    if (!c) return;
    if (c->stream || c->cap_stream) cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    while (!c->allocs.empty()) dev_free(c, c->allocs.back().p);
    for (int i = 0; i < snn_ctx::kStageBufs; ++i) {
        if (c->stage_ev[i]) cudaEventDestroy(c->stage_ev[i]);
        if (c->stage[i]) cudaFreeHost(c->stage[i]);
    }
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->side) cudaStreamDestroy(c->side);
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    cudaGetLastError();
    delete c;
}

}  // extern "C"
