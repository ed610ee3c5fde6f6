"""Benchmark: synaptic events/s and realtime factor of the work-queue SNN
timestep on one B300 (or N, one process per GPU).

Default workload: the batched sweep of 256 independent Brunel networks
(1,000-50,000 neurons, log-uniform; in-degree 10 % capped at 1,000;
g ~ U[3,7]; nu_ext/nu_thr ~ U[0.9,4]; 15-step delay) with 16-bit weights,
all stepped together.  One bench "step" is one simulation timestep of every
network (Update Neurons -> delay FIFO -> Receive Spikes).  The same line
reports the plain binary32-weight path with the global-atomic receive on
the same networks, the roofline of the dominant kernel, the end-to-end rate
through the C ABI from host buffers, and the CPU oracle on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import snn_inputs as si  # noqa: E402

DT_MS = 0.1
METRIC = "synaptic events/s and realtime factor on 1 B300, batched+int16 vs plain FP32"
# algorithmic bytes (what the method must move): per delivered event the
# edge as the receive stores it -- a 4-byte target and a 2-byte (int16) or
# 4-byte (binary32) weight, or one 4-byte packed edge (16-bit target offset
# in its instance, int16 code; the library reports which); per
# delivered spike its two row offsets (16 B) and its queue entry (4 B); per
# emitted spike the queue write (4 B) and the log entry (8 B); per neuron and
# step the state the update reads and writes (Brunel: V 4+4, refractory 1+1,
# input 4 read + 4 cleared = 18 B; Vogels 44 B; STDP traces +16 B).
B_SPIKE_DELIVERED, B_SPIKE_EMITTED = 20, 12
B_ROW_WEIGHT = 4  # per delivered spike, when the receive reads its row's one weight


def reads_row_weights(info: dict) -> bool:
    """The receive takes each row's one weight from a per-row array (16-bit
    target offsets in the tiled receive, 4-byte targets in the global one)."""
    return info["edge_bytes"] == 2 or (info["receive"] == "global" and info["edge_bytes"] == 4)


def spike_bytes(info: dict) -> int:
    """Bytes per delivered spike: row offsets 16 + queue entry 4 (+ row weight)."""
    return B_SPIKE_DELIVERED + (B_ROW_WEIGHT if reads_row_weights(info) else 0)
B_NEURON = {si.BRUNEL: 18, si.VOGELS: 44}
B_NEURON_STDP = 16


def gpu_launches(steps: int, recv_kind: str, stdp: bool, lazy: bool = False, per_graph: int = 16,
                 fused: bool = False, persistent: bool = False) -> int:
    """Kernels of this library launched by one snn_step call of `steps` steps:
    the update, the STDP passes (eager: depression and potentiation; lazy: one
    replay pass), the receive (tiled: per-step plan and receive; bulk:
    receive, merge; global: receive) -- or the one fused step kernel -- and
    one step-counter advance per captured graph (per_graph steps, the rest one
    by one); the persistent form launches once per call."""
    if persistent:
        return 1
    if fused:
        per_step = 1
    else:
        per_step = 1 + ((1 if lazy else 2) if stdp else 0) + {"tiled": 2, "bulk": 2, "global": 1}[recv_kind]
    return steps * per_step + steps // per_graph + steps % per_graph


# the sources each ncu traffic summary depends on (profiles/<file>)
TRAFFIC_FILES = {"k_receive_tiled": ("receive_traffic.txt", ("snn_tiled.cuh", "snn_device.cuh")),
                 "k_step_fused": ("fused_step_traffic.txt",
                                  ("snn_fused.cuh", "snn_tiled.cuh", "snn_kernels.cuh", "snn_device.cuh"))}


def kernel_source_hash(kernel: str = "k_receive_tiled") -> str:
    """Hash of the sources of a kernel (its ncu traffic figure is only
    reported while these are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    for f in TRAFFIC_FILES[kernel][1]:
        with open(os.path.join(ROOT, "paper_1912_07423_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_ratio(kernel: str = "k_receive_tiled"):
    """DRAM bytes per algorithmic byte of a kernel from its committed ncu
    summary under profiles/, if that summary matches the sources."""
    try:
        kv = {}
        with open(os.path.join(ROOT, "profiles", TRAFFIC_FILES[kernel][0])) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_hash") != kernel_source_hash(kernel):
            return None
        return float(kv["dram_bytes_per_algorithmic_byte"])
    except Exception:
        return None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def replica_seed(rank: int) -> int:
    """Graph seed base of the replica on `rank` (each rank simulates its own
    networks: weak scaling, no data-path collective)."""
    return 1 + 1000 * rank


def workload(name: str, rank: int):
    if name == "batched_sweep_256":
        return si.batched_sweep(256, base_seed=replica_seed(rank), n_steps=0)
    if name.startswith("batched_sweep_"):  # a smaller sweep of the same recipe (profiling)
        return si.batched_sweep(int(name.rsplit("_", 1)[1]), base_seed=replica_seed(rank), n_steps=0)
    if name == "vogels_1m":
        return si.vogels_1m(seed=1 + rank, n_steps=0)
    if name == "brunel_12k5":
        return si.brunel_12k5(seed=1 + rank, n_steps=0)
    if name == "vogels_4k":
        return si.vogels_4k(seed=1 + rank, n_steps=0)
    if name == "brunel_stdp_100k":
        return si.brunel_stdp_100k(seed=1 + rank, n_steps=0)
    raise SystemExit(f"unknown workload {name}")


def oracle_sample(prob, max_neurons=170_000, max_inst=12):
    """A deterministic sample of the workload the oracle can step in
    milliseconds: its first instances (or the whole problem if small)."""
    if len(prob.instances) == 1:
        return prob, "the whole network"
    b, n = 0, 0
    while b < min(max_inst, len(prob.instances)) and n + prob.instances[b].n <= max_neurons:
        n += prob.instances[b].n
        b += 1
    b = max(b, 1)
    lo, hi = 0, int(prob.inst_off[b])
    e1 = int(prob.row_off[hi])
    sub = si.Problem(model=prob.model, instances=prob.instances[:b], delay=prob.delay, seed=prob.seed, n_steps=0,
                     stdp=prob.stdp, inst_off=prob.inst_off[:b + 1].copy(), row_off=prob.row_off[:hi + 1].copy(),
                     tgt=prob.tgt[:e1], w=prob.w[:e1])
    return sub, f"instances 0-{b - 1} of the sweep ({n} neurons, {e1} synapses)"


def sweep_size(name: str) -> int:
    """Networks of a batched-sweep workload (0 for the single networks)."""
    return int(name.rsplit("_", 1)[1]) if name.startswith("batched_sweep_") else 0


def _oracle_window_process(base_seed, n_nets, b, t0, k_min, target_s, per_step, barrier, out):
    """One process of the oracle sample: network b of the sweep, rebuilt alone
    (same graph and Philox keys as inside the batch), timed on the window of
    steps [t0, t0 + k) as the difference of two runs from step 0, to t0 + k
    and to t0 (the oracle always starts at step 0).  With target_s, a
    200-step calibration run of every process goes to the shared per_step
    array, and all processes take the same k: the one that gives the slowest
    network's longer run about target_s seconds (at least k_min)."""
    try:
        import oracle
        inst = si.batched_sweep_params(n_nets, base_seed)[b]
        p = si.problem(si.BRUNEL, [inst], delay=15, n_steps=200, seed=base_seed, threads=1, inst_index0=b)
        if target_s:
            c0 = time.perf_counter()
            oracle.run(p, inst_key0=b)
            per_step[b] = (time.perf_counter() - c0) / 200
        barrier.wait(timeout=900)
        k = k_min
        if target_s:
            k = int(max(k_min, target_s / max(max(per_step[:]), 1e-7) - t0))
        p.n_steps = t0
        a0 = time.perf_counter()
        ra = oracle.run(p, inst_key0=b)
        a1 = time.perf_counter()
        p.n_steps = t0 + k
        rb = oracle.run(p, inst_key0=b)
        b1 = time.perf_counter()
        out.put((b, k, int(rb["events"]) - int(ra["events"]), (b1 - a1) - (a1 - a0), p.n_edges, inst.n))
    except Exception as e:  # reported to the parent, which falls back to one process
        barrier.abort()
        out.put((b, -1, 0, 0.0, repr(e), 0))


def oracle_window(name: str, rank: int, t0: int, k_min: int, target_s: float | None, timeout_s: float = 1800.0):
    """The oracle on the first networks of a batched sweep, one single-threaded
    process per host core (as many as the free host memory holds), started
    together behind a barrier, each timed on steps [t0, t0 + k) of its
    network.  The value is the sum of the per-process rates (each process has
    a core of its own).  Returns (events/s, cores, description, seconds, k,
    per-process (network, k, events, seconds)) or None if a process failed."""
    import multiprocessing as mp
    import queue
    n_nets = sweep_size(name)
    base = replica_seed(rank)
    params = si.batched_sweep_params(n_nets, base)
    cores = len(os.sched_getaffinity(0))
    free = os.sysconf("SC_AVPHYS_PAGES") * os.sysconf("SC_PAGE_SIZE")
    k, need = 0, 0
    while k < min(cores, n_nets):
        e = params[k].n * (params[k].k_exc + params[k].k_inh)
        cost = 32 * e + 512 * params[k].n + (256 << 20)  # graph copies (about 13 B per edge measured), state, interpreter
        if k > 0 and need + cost > free // 2:
            break
        need += cost
        k += 1
    ctx = mp.get_context("spawn")  # a fresh interpreter per process: safe beside a CUDA context
    barrier, out, per_step = ctx.Barrier(k), ctx.Queue(), ctx.Array("d", k)
    procs = [ctx.Process(target=_oracle_window_process,
                         args=(base, n_nets, b, t0, k_min, target_s, per_step, barrier, out), daemon=True)
             for b in range(k)]
    for pr in procs:
        pr.start()
    res, deadline = [], time.monotonic() + timeout_s
    while len(res) < k and time.monotonic() < deadline:
        try:
            res.append(out.get(timeout=5.0))
        except queue.Empty:  # a process that died without reporting ends the sample
            if any(pr.exitcode not in (None, 0) for pr in procs):
                barrier.abort()
                break
    for pr in procs:
        pr.join(timeout=10)
        if pr.is_alive():
            pr.kill()
    if len(res) != k or any(r[1] < 0 for r in res):
        why = [r[4] for r in res if r[1] < 0] or [f"{k - len(res)} of {k} processes did not report"]
        print(f"parallel oracle sample failed ({why[0]}); timing one process instead", file=sys.stderr)
        return None
    value = sum(r[2] / r[3] for r in res if r[3] > 0)
    ks = sorted(r[1] for r in res)
    secs = max(r[3] for r in res)
    desc = (f"networks 0-{k - 1} of the sweep, one single-threaded C oracle process each on {k} host cores "
            f"({sum(r[5] for r in res)} neurons, {sum(r[4] for r in res)} synapses), steps [{t0}, {t0 + ks[0]}) "
            f"(at least {k_min} steps), each process timed as the difference of two runs from step 0; "
            f"value = sum of the per-process rates")
    return value, k, desc, secs, ks[0], sorted((r[0], r[1], r[2], r[3]) for r in res)


def oracle_window_single(prob, t0: int, k_min: int, target_s: float | None):
    """The oracle, single-threaded, on a sample of a non-sweep workload
    (oracle_sample), timed on steps [t0, t0 + k) as the difference of two runs
    from step 0."""
    import oracle
    sub, desc = oracle_sample(prob)
    k = k_min
    if target_s:
        sub.n_steps = 200
        c0 = time.perf_counter()
        oracle.run(sub)
        per_step = (time.perf_counter() - c0) / 200
        k = int(max(k_min, target_s / max(per_step, 1e-7) - t0))
    sub.n_steps = t0
    a0 = time.perf_counter()
    ra = oracle.run(sub)
    a1 = time.perf_counter()
    sub.n_steps = t0 + k
    rb = oracle.run(sub)
    b1 = time.perf_counter()
    dt = (b1 - a1) - (a1 - a0)
    ev = int(rb["events"]) - int(ra["events"])
    return (ev / dt, 1, f"{desc}, steps [{t0}, {t0 + k}) timed as the difference of two runs from step 0, "
            "single-threaded C oracle", dt, k, [(0, k, ev, dt)])


def cpu_window(name: str, prob, rank: int, t0: int, k_min: int, target_s: float | None):
    """The oracle timed on the GPU's window: the parallel sweep sample, or one
    process (also the fallback when the parallel sample fails)."""
    r = oracle_window(name, rank, t0, k_min, target_s) if sweep_size(name) else None
    if r is None:
        if prob is None:
            prob = workload(name, rank)
        r = oracle_window_single(prob, t0, k_min, target_s)
    return r


def cpu_baseline(prob, t0: int, steps: int, target_s: float = 15.0, name: str = "", rank: int = 0):
    """The CPU oracle on the host cores, on the same window of steps as the
    GPU's timed region (at least 100 steps of it), sized to about target_s
    seconds per process."""
    value, cores, desc, secs, k, _ = cpu_window(name, prob, rank, t0, max(steps, 100), target_s)
    return {"value": value, "unit": "synaptic events/s", "cores": cores, "kind": "oracle", "sample": desc,
            "seconds": round(secs, 3), "window": [t0, t0 + k]}


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons every 50 ms,
    summarised over a span of host time (the device work of the run)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        # raw samples (the JSON line carries their summary); SNN_CLOCKS_DIR keeps them elsewhere
        import tempfile
        self.path = os.path.join(os.environ.get("SNN_CLOCKS_DIR", tempfile.gettempdir()), f"snn_clocks_rank{index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    @staticmethod
    def _when(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def stop(self, t_from: float | None = None, t_to: float | None = None):
        """Stop sampling; summarise the samples taken between host times
        t_from and t_to (time.time(); all samples if not given)."""
        if not self.proc:
            return None
        time.sleep(0.1)  # the sample in flight
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, n_all = [], [], set(), 0
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 10:
                continue
            n_all += 1
            w = self._when(parts[0])
            if t_from is not None and w is not None and not (t_from - 0.05 <= w <= t_to + 0.05):
                continue
            try:
                sm.append(float(parts[2]))
                mx.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[6:10]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "span_s": None if t_from is None else round(t_to - t_from, 3),
                "span": "from the network's creation to the end of the profiled steps"}


def delivered_spikes(net, prob, t0: int, t1: int) -> int:
    """Spikes delivered by the receives of steps [t0, t1) (queue S_{t-d+1})."""
    a, b = max(0, t0 - prob.delay + 1), max(0, t1 - prob.delay + 1)
    if b <= a:
        return 0
    steps, _ = net.spikes(a, b)
    return len(steps)


def graph_construction(prob, dev, hbm: float, reps: int = 3) -> dict:
    """snn_expand_jobs (Fig. 2) with one job per neuron of the workload: n =
    its out-degree, values from its own instance's id range, written at its
    row offset -- the workload's adjacency, built on the device.  One
    warm-up call, then reps calls timed with CUDA events on the stream (each
    call also waits for its error flag).  Algorithmic bytes: 4 per value
    written + 24 per job record read."""
    import torch
    import paper_1912_07423_b300 as snn
    deg = np.diff(prob.row_off.astype(np.int64)).astype(np.uint32)
    inst_of = np.repeat(np.arange(len(prob.instances)), np.diff(prob.inst_off.astype(np.int64)))
    jobs = np.zeros(prob.n, dtype=snn.JOB_DTYPE)
    jobs["n"] = deg
    jobs["a"] = prob.inst_off[inst_of]
    jobs["b"] = prob.inst_off[inst_of + 1]
    jobs["o"] = prob.row_off[:-1]
    djobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    E = int(prob.row_off[-1])
    buf = torch.empty(E, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    snn.expand_jobs(djobs, 1, E, out=buf)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        snn.expand_jobs(djobs, 1, E, out=buf)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3 / reps
    nbytes = 4.0 * E + 24.0 * prob.n
    del buf, djobs
    torch.cuda.empty_cache()
    return {"values": E, "jobs": int(prob.n), "seconds": t, "values_per_s": E / t,
            "achieved_gbs": nbytes / t / 1e9, "frac_of_hbm": nbytes / t / 1e9 / hbm,
            "what": "snn_expand_jobs: one job per neuron (out-degree values from its instance's ids)"}


def launch_bytes(net, prob, t0: int, n: int, edge_bytes: int, per_spike: int = B_SPIKE_DELIVERED) -> list:
    """Algorithmic bytes of the receive launches of steps t0 .. t0+n-1, from
    the spike log and the row lengths: the receive of step t delivers the
    spikes of step t+1-d, each a whole row (an ncu capture of one of these
    launches compares with its entry)."""
    a = max(0, t0 - prob.delay + 1)
    steps, ids = net.spikes(a, a + n)
    deg = np.diff(prob.row_off.astype(np.int64))
    out = []
    for t in range(t0, t0 + n):
        m = steps == t + 1 - prob.delay
        out.append(int(deg[ids[m]].sum()) * edge_bytes + int(m.sum()) * per_spike)
    return out


def step_bytes(prob, edge_bytes: int, events: int, delivered: int, emitted: int, steps: int,
               per_spike: int = B_SPIKE_DELIVERED) -> float:
    per_neuron = B_NEURON[prob.model] + (B_NEURON_STDP if prob.stdp else 0)
    return (events * edge_bytes + delivered * per_spike +
            emitted * B_SPIKE_EMITTED + per_neuron * prob.n * steps)


def reduce_over_ranks(x: float, op: str, dist, device) -> float:
    """x combined over the ranks ("max": the slowest rank's time, "sum": the
    job's events); dist is torch.distributed or None (one rank), device the
    tensor device of the process group's backend (cuda for NCCL, cpu for gloo)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_value(events: float, seconds: float, dist, device) -> float:
    """Whole-job throughput of weakly scaled replicas: the events of all ranks
    over the slowest rank's time."""
    return reduce_over_ranks(events, "sum", dist, device) / reduce_over_ranks(seconds, "max", dist, device)


def isi_stats(steps, ids, n: int, t0: int, t1: int, dt_ms: float):
    """Population rate (Hz) and mean ISI CV of a raster over steps [t0, t1),
    with the definitions of snn_stats: rate = spikes / n / window; CV per
    neuron with at least 3 spikes in the window (ISIs between its consecutive
    spikes there), averaged over those neurons."""
    m = (steps >= t0) & (steps < t1)
    st, i = steps[m].astype(np.int64), ids[m].astype(np.int64)
    rate = len(st) / n / ((t1 - t0) * dt_ms * 1e-3)
    order = np.lexsort((st, i))
    st, i = st[order], i[order]
    cnt = np.bincount(i, minlength=n)
    same = i[1:] == i[:-1]
    isi = (st[1:] - st[:-1])[same].astype(np.float64)
    who = i[1:][same]
    s1 = np.bincount(who, weights=isi, minlength=n)
    s2 = np.bincount(who, weights=isi * isi, minlength=n)
    ok = cnt >= 3
    if not ok.any():
        return rate, 0.0
    mean = s1[ok] / (cnt[ok] - 1)
    var = s2[ok] / (cnt[ok] - 1) - mean * mean
    return rate, float((np.sqrt(np.maximum(var, 0.0)) / mean).mean())


def _f64_stats(sub, key0: int, t0: int, t1: int, dt_ms: float):
    import oracle
    sub.n_steps = t1
    r = oracle.run_f64(sub, inst_key0=key0)
    return isi_stats(r["steps"], r["ids"], sub.n, t0, t1, dt_ms)


def drift_networks(prob) -> list:
    """Networks of the workload whose rate and ISI CV are compared with the
    binary64 oracle: for a batch the ones at the 25/50/75 % size quantiles and
    the largest; a single network whole if the oracle holds it (<= 200k neurons)."""
    B = len(prob.instances)
    if B == 1:
        return [0] if prob.n <= 200_000 and not prob.stdp else []
    order = sorted(range(B), key=lambda b: prob.instances[b].n)
    return sorted({order[int(q * (B - 1))] for q in (0.25, 0.5, 0.75, 1.0)})


def rate_cv_drift(prob, t0: int, k: int, device) -> dict | None:
    """Rate and ISI CV of the binary32 lattice run on the GPU (snn_stats over
    steps [t0, t0 + k), each sampled network re-run alone in its own context
    with its batch key, hence bit-identical to its part of the batch) against
    the binary64, unquantised-weight oracle of the same networks and window
    (run in host processes while the GPU runs).  Bounds: rate within 2 %,
    ISI CV within 5 %, of the pooled values."""
    import concurrent.futures as cf
    import multiprocessing as mp
    import paper_1912_07423_b300 as snn
    nets = drift_networks(prob)
    if not nets:
        return None
    dt_ms = prob.instances[0].dt
    subs = [si.sub_problem(prob, b, n_steps=0) if len(prob.instances) > 1 else prob for b in nets]
    keys = nets if len(prob.instances) > 1 else [0]
    with cf.ProcessPoolExecutor(max_workers=min(len(nets), max(1, len(os.sched_getaffinity(0)))),
                                mp_context=mp.get_context("spawn")) as ex:
        futs = [ex.submit(_f64_stats, dataclasses.replace(sub), key, t0, t0 + k, dt_ms) for sub, key in zip(subs, keys)]
        gpu = []
        for sub, key in zip(subs, keys):
            with snn.Network(sub, w16=True, stats=True, inst_key0=key, log_capacity=0) as net:
                net.step(t0)
                net.stats_clear()
                net.step(k)
                gpu.append(net.stats(0))
        f64 = [f.result() for f in futs]
    n = [sub.n for sub in subs]
    pool = lambda xs: sum(x * w for x, w in zip(xs, n)) / sum(n)  # neuron-weighted
    r32, r64 = pool([g[0] for g in gpu]), pool([f[0] for f in f64])
    c32, c64 = sum(g[1] for g in gpu) / len(gpu), sum(f[1] for f in f64) / len(f64)
    dr, dc = abs(r32 - r64) / r64 if r64 else 0.0, abs(c32 - c64) / c64 if c64 else 0.0
    return {"networks": nets, "window": [t0, t0 + k],
            "gpu_rate_hz": r32, "f64_rate_hz": r64, "rate_rel_diff": dr,
            "gpu_isi_cv": c32, "f64_isi_cv": c64, "isi_cv_rel_diff": dc,
            "within_bounds": bool(dr <= 0.02 and dc <= 0.05), "bounds": {"rate": 0.02, "isi_cv": 0.05},
            "per_network": [{"net": b, "gpu": list(g), "f64": list(f)} for b, g, f in zip(nets, gpu, f64)]}


def run_ours(args, rank, world, dist):
    import torch
    import paper_1912_07423_b300 as snn

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    clocks = ClockSampler(dev.index)
    clocks.start()  # running before the device work starts: it spans settle, warm-up, timed and profiled steps
    t_gen = time.perf_counter()
    prob = workload(args.workload, rank)
    t_gen = time.perf_counter() - t_gen
    hbm, peak_kind = peaks()
    t0 = args.settle + args.warmup  # first timed step
    cap = int(prob.n * (t0 + args.steps) * 0.05) + (1 << 20)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_over_ranks(x, "max", dist, dev)

    def sum_over_ranks(x: float) -> float:
        return reduce_over_ranks(x, "sum", dist, dev)

    def timed(net, steps):
        stream = net.stream
        c0 = net.counters()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        net.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        barrier()
        net.sync()
        c1 = net.counters()
        return e0.elapsed_time(e1) / 1e3, c1["events"] - c0["events"], c1["spikes"] - c0["spikes"]

    # ---- headline: batched + int16, timed on the device over steps [t0, t0 + K)
    recv_mode = {"auto": snn.RECV_AUTO, "global": snn.RECV_GLOBAL, "tiled": snn.RECV_TILED,
                 "bulk": snn.RECV_BULK, "persistent": snn.RECV_PERSISTENT}[args.receive]
    lazy = prob.stdp and args.plasticity == "lazy"
    t_clk0 = time.time()
    net = snn.Network(prob, w16=True, receive=recv_mode, log_capacity=cap, lazy=lazy, lazy_fifo=args.lazy_fifo,
                      serial=args.serial)
    info = net.info()
    recv_kind = info["receive"]
    net.step(args.settle)  # the initial transient passes and the delay FIFO fills
    net.step(args.warmup)
    net.sync()
    t_main, ev_main, sp_main = timed(net, args.steps)
    deliv_main = delivered_spikes(net, prob, t0, t0 + args.steps)
    # ---- the same window again from a reset, with CUDA events around every
    # kernel (deterministic: the same spikes and events as the timed steps)
    n_prof = args.steps if args.profile_steps <= 0 else min(args.steps, args.profile_steps)
    net.reset()
    net.step(t0)
    net.sync()
    c0 = net.counters()
    phases = net.step_profiled(n_prof)
    c1 = net.counters()
    clk = clocks.stop(t_clk0, time.time())
    bytes_each = launch_bytes(net, prob, t0, min(n_prof, 16), info["edge_bytes"], spike_bytes(info))
    ev_p, sp_p = c1["events"] - c0["events"], c1["spikes"] - c0["spikes"]
    deliv_p = delivered_spikes(net, prob, t0, t0 + n_prof)
    mem = info["device_bytes"]
    net.close()
    del net
    torch.cuda.empty_cache()

    t_max = max_over_ranks(t_main)
    ev_total = sum_over_ranks(ev_main)
    value = ev_total / t_max
    fused = bool(info.get("fused"))
    persistent = bool(info.get("persistent"))
    # the dominant kernel: the receive, or the fused step kernel or the
    # persistent launch, which also run the update (their bytes: the
    # receive's plus the update's per-neuron state and per-emitted-spike
    # queue and log writes)
    kernel = "k_step_fused" if fused else ("k_persistent" if persistent else f"k_receive_{recv_kind}")
    recv_ms = phases["receive"] / n_prof
    upd_bytes = ((B_NEURON[prob.model] * prob.n * n_prof + B_SPIKE_EMITTED * sp_p) / n_prof
                 if fused or persistent else 0.0)
    sb = spike_bytes(info)
    recv_bytes = (ev_p * info["edge_bytes"] + deliv_p * sb) / n_prof + upd_bytes
    achieved = recv_bytes / (recv_ms * 1e-3) / 1e9

    def frac_at(edge_b: int, spike_b: int) -> float:
        """The kernel's fraction of the measured HBM rate had its events been
        stored at edge_b bytes each (same time, same events and spikes)."""
        b = (ev_p * edge_b + deliv_p * spike_b) / n_prof + upd_bytes
        return b / (recv_ms * 1e-3) / 1e9 / hbm
    step_b = step_bytes(prob, info["edge_bytes"], ev_main, deliv_main, sp_main, args.steps, sb)
    step_frac = (step_b / (hbm * 1e9)) / t_main

    out = {"metric": METRIC, "value": value, "unit": "synaptic events/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int16 weights, int32 input, f32 state",
           "data": "synthetic (seeded graphs, no dataset)",
           "config": {"workload": args.workload, "networks": len(prob.instances), "neurons": prob.n,
                      "synapses": prob.n_edges, "delay_steps": prob.delay, "dt_ms": DT_MS,
                      "window": [t0, t0 + args.steps], "settle_steps": args.settle,
                      "receive": recv_kind, "tiles": info["n_tiles"], "weights": "int16 x 2^shift(row)",
                      "step_kernels": ("fused (update + receive in one kernel)" if fused else
                                       ("persistent (one cooperative launch per call, %d CTAs)" % info["persist_ctas"]
                                        if persistent else "separate")),
                      **({"tuned_ms_per_step": {k: v for k, v in info["tune_ms"].items() if v > 0}}
                         if info.get("tuned") else {}),
                      "edge_bytes": info["edge_bytes"],
                      "l2": "inputs larger than L2 (edge arrays %.1f GB >> 126 MB)" % (prob.n_edges * 6 / 1e9),
                      "parallelism": f"replicas x{world} (independent networks, no collective)",
                      "graph_gen_s": round(t_gen, 1), "device_bytes": mem,
                      **({"plasticity": ("lazy, history %d steps" % (args.lazy_fifo or 128)) if lazy else "eager"}
                         if prob.stdp else {})},
           "realtime_factor": args.steps * DT_MS * 1e-3 / t_max,
           "spikes": int(sp_main), "events": int(ev_main),
           "roofline": {"kernel": kernel, "bound": "hbm", "achieved": achieved, "peak": hbm,
                        "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": (traffic_ratio(kernel) * recv_bytes
                                    if kernel in TRAFFIC_FILES and traffic_ratio(kernel) else None),
                        "update_bytes_per_launch": upd_bytes,
                        "launch_ms": recv_ms,
                        "bytes_per_launch": recv_bytes, "launches": n_prof,
                        "window": [t0, t0 + n_prof],
                        "same_events_as_timed": bool(n_prof == args.steps and ev_p == ev_main),
                        "bytes_each": bytes_each[:16],
                        "edge_bytes": info["edge_bytes"], "spike_bytes": sb,
                        # the same time and events measured against other edge layouts: a 4-byte
                        # target per synapse (the paper's Table 2 layout for Vogels / Brunel) and a
                        # 4-byte target + 2-byte weight code
                        "frac_at_4_bytes_per_event": frac_at(4, B_SPIKE_DELIVERED),
                        "frac_at_6_bytes_per_event": frac_at(6, B_SPIKE_DELIVERED),
                        "events_per_s_in_kernel": ev_p / n_prof / (recv_ms * 1e-3),
                        # effective bytes per delivered event (edges + per-spike records) and the
                        # events/s the measured HBM rate allows for the edges alone
                        "bytes_per_event": recv_bytes * n_prof / max(ev_p, 1),
                        "edge_only_ceiling_events_per_s": hbm * 1e9 / info["edge_bytes"]},
           "step_roofline": {"bytes_per_step": step_b / args.steps, "frac": step_frac, "peak": hbm,
                             "unit": "GB/s", "achieved": step_b / t_main / 1e9,
                             "bytes_per_event": step_b / max(ev_main, 1)},
           "phase_ms_per_step": {k: v / n_prof for k, v in phases.items()},
           "gpu_launches": gpu_launches(args.steps, recv_kind, prob.stdp, lazy, fused=fused, persistent=persistent),
           "clocks": clk}

    # ---- the same path with Update Neurons and Receive Spikes as separate
    # kernels (SNN_F_SERIAL), same window: what running them in one kernel gains
    if fused and not args.no_serial_compare:
        with snn.Network(prob, w16=True, receive=recv_mode, log_capacity=cap, serial=True) as snet:
            snet.step(t0)
            snet.sync()
            t_s, ev_s, sp_s = timed(snet, args.steps)
        torch.cuda.empty_cache()
        out["separate_kernels"] = {"value": sum_over_ranks(ev_s) / max_over_ranks(t_s), "unit": "synaptic events/s",
                                   "ms_per_step": t_s * 1e3 / args.steps,
                                   "same_events_and_spikes": bool(ev_s == ev_main and sp_s == sp_main)}
        out["speedup_fused_vs_separate"] = out["value"] / out["separate_kernels"]["value"]

    # ---- plain path: binary32 weights, global-atomic receive, each network in
    # its own context one after the other (its batch key: the same spikes)
    if not args.no_plain:
        t_pl, ev_pl, n_ctx = 0.0, 0, 0
        B = len(prob.instances)
        for b in range(B):
            sub = si.sub_problem(prob, b, n_steps=0) if B > 1 else prob
            with snn.Network(sub, w16=False, receive=snn.RECV_GLOBAL, log_capacity=0, lazy=lazy,
                             lazy_fifo=args.lazy_fifo, inst_key0=b if B > 1 else 0) as pnet:
                pnet.step(t0)
                pnet.sync()
                t_b, ev_b, _ = timed(pnet, args.steps)
            t_pl += t_b
            ev_pl += ev_b
            n_ctx += 1
        torch.cuda.empty_cache()
        out["plain_fp32"] = {"value": sum_over_ranks(ev_pl) / max_over_ranks(t_pl), "unit": "synaptic events/s",
                             "receive": "global", "weights": "binary32",
                             "contexts": n_ctx, "how": "each network alone in its own context, one after another; "
                                                        "time = sum of the per-network CUDA-event times",
                             "same_events": bool(ev_pl == ev_main),
                             "ms_per_step": t_pl * 1e3 / args.steps,
                             "realtime_factor": args.steps * DT_MS * 1e-3 / t_pl}
        out["speedup_vs_plain_fp32"] = out["value"] / out["plain_fp32"]["value"]

    # ---- the same networks through the generic update (Section III-B): Brunel
    # written as a specialisation of the LIF building block
    if not args.no_generic and prob.model == si.BRUNEL and not prob.stdp:
        gprob = dataclasses.replace(prob, model=snn.MODEL_BRUNEL_LIF)
        net = snn.Network(gprob, w16=True, receive=recv_mode, log_capacity=cap)
        net.step(t0)
        net.sync()
        t_g, ev_g, sp_g = timed(net, args.steps)
        net.close()
        del net
        torch.cuda.empty_cache()
        out["generic_update"] = {"value": sum_over_ranks(ev_g) / max_over_ranks(t_g), "unit": "synaptic events/s",
                                 "ms_per_step": t_g * 1e3 / args.steps,
                                 "model": "Brunel from the LIF building block (SNN_MODEL_BRUNEL_LIF)",
                                 "same_events_and_spikes": bool(ev_g == ev_main and sp_g == sp_main)}

    # ---- end to end through the C ABI from host buffers: create + graph
    # upload, the steps up to the end of the window, raster readout
    if not args.no_e2e:
        barrier()
        torch.cuda.synchronize()
        t_s = time.perf_counter()
        net = snn.Network(prob, w16=True, receive=recv_mode, log_capacity=cap, lazy=lazy,
                          lazy_fifo=args.lazy_fifo)  # h2d of the graph
        t1 = time.perf_counter()
        net.step(t0 + args.steps)
        net.sync()
        t2 = time.perf_counter()
        steps_h, ids_h = net.spikes()  # d2h of the raster
        t_e2e = time.perf_counter() - t_s
        parts = {"create_and_build_s": t1 - t_s, "steps_s": t2 - t1, "raster_readout_s": t_s + t_e2e - t2}
        c = net.counters()
        net.close()
        del net
        torch.cuda.empty_cache()
        n_all = t0 + args.steps
        w_row = prob.row_weights()  # the Network above loaded the graph from one weight per row when it could
        h2d = prob.row_off.nbytes + prob.tgt.nbytes + (w_row.nbytes if w_row is not None else prob.w.nbytes)
        d2h = 8 * int(c["spikes"])
        out["e2e"] = {"value": sum_over_ranks(c["events"]) / max_over_ranks(t_e2e), "unit": "synaptic events/s",
                      "seconds": t_e2e, "steps": n_all, "h2d_bytes_per_step": h2d / n_all,
                      "d2h_bytes_per_step": d2h / n_all,
                      "includes": "snn_create + " + ("snn_build_graph_rows (targets, one weight per row)" if w_row is not None
                                                     else "snn_build_graph (targets, weight per synapse)")
                                  + " from host arrays + snn_step(settle + warm-up + K) + snn_read_spikes",
                      "parts": parts}

    # ---- binary32 lattice run against the binary64 float-weight oracle
    if not args.no_drift and rank == 0:
        out["rate_cv_drift"] = rate_cv_drift(prob, t0, max(args.steps, args.drift_steps), dev)

    # ---- adjacency construction on the GPU (Fig. 2) for the same networks
    if not args.no_graph:
        out["graph_construction"] = graph_construction(prob, dev, hbm)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the baseline is a one-GPU figure
        out["cpu_baseline"] = cpu_baseline(prob, t0, args.steps, name=args.workload, rank=rank)
    return out


def run_reference(args, rank):
    """The oracle, as it stands, on a bounded sample of the same workload, on
    the host cores, timed on the same window of steps as our arm (at least 100
    steps of it, from t0 = settle + warm-up)."""
    t0 = args.settle + args.warmup
    value, cores, desc, dt, k, _ = cpu_window(args.workload, None, rank, t0, max(args.steps, 100), args.ref_seconds)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "synaptic events/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / k,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, int32 input",
            "data": "synthetic (seeded graphs, no dataset)",
            "config": {"workload": args.workload, "window": [t0, t0 + k], "settle_steps": args.settle,
                       "sample": desc},
            "cpu_baseline": {"value": value, "unit": "synaptic events/s", "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": "synaptic events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="batched_sweep_256")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="steps of the timed window profiled again from a reset (0: all of --steps)")
    ap.add_argument("--settle", type=int, default=200,
                    help="untimed steps before the warm-up: the initial transient passes and the delay FIFO fills")
    ap.add_argument("--drift-steps", type=int, default=2000, help="window of the rate / ISI CV drift comparison")
    ap.add_argument("--ref-seconds", type=float, default=15.0,
                    help="reference arm: about this long per process on the host cores")
    ap.add_argument("--receive", choices=["auto", "global", "tiled", "bulk", "persistent"], default="auto")
    ap.add_argument("--plasticity", choices=["eager", "lazy"], default="eager",
                    help="Update Synapses form for plastic workloads (brunel_stdp_100k; eager measured faster)")
    ap.add_argument("--lazy-fifo", type=int, default=0, help="lazy plasticity: history length (0: 128)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-generic", action="store_true", help="skip timing the generic-update model")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip timing the GPU adjacency construction")
    ap.add_argument("--no-drift", action="store_true", help="skip the binary64 rate / ISI CV comparison")
    ap.add_argument("--no-serial-compare", action="store_true",
                    help="skip timing the separate update and receive kernels beside the fused step")
    ap.add_argument("--serial", action="store_true",
                    help="headline with Update Neurons and Receive Spikes as separate kernels (SNN_F_SERIAL)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    if args.settle < 0:
        raise SystemExit("--settle must be >= 0")
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args, rank)), flush=True)
        return

    dist = None
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
        tdist.init_process_group("nccl")
        dist = tdist
    out = run_ours(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
