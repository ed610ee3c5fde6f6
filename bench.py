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
B_NEURON = {si.BRUNEL: 18, si.VOGELS: 44}
B_NEURON_STDP = 16


def gpu_launches(steps: int, recv_kind: str, stdp: bool, lazy: bool = False, per_graph: int = 16) -> int:
    """Kernels of this library launched by `steps` steps of snn_step: the
    update, the STDP passes (eager: depression and potentiation; lazy: one
    replay pass), the receive (tiled: per-step plan and receive; bulk:
    receive, merge; global: receive), and one step-counter advance per
    captured graph (per_graph steps, the rest one by one)."""
    per_step = 1 + ((1 if lazy else 2) if stdp else 0) + {"tiled": 2, "bulk": 2, "global": 1}[recv_kind]
    return steps * per_step + steps // per_graph + steps % per_graph

def kernel_source_hash() -> str:
    """Hash of the sources of the tiled receive (its ncu traffic figure is
    only reported while these are unchanged)."""
    import hashlib
    h = hashlib.sha256()
    for f in ("snn_tiled.cuh", "snn_device.cuh"):
        with open(os.path.join(ROOT, "paper_1912_07423_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_ratio():
    """DRAM bytes per algorithmic byte of k_receive_tiled from the committed
    ncu summary (profiles/receive_traffic.txt), if it matches the sources."""
    try:
        kv = {}
        with open(os.path.join(ROOT, "profiles", "receive_traffic.txt")) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_hash") != kernel_source_hash():
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


def _oracle_process(base_seed, n_nets, b, steps, target_s, barrier, out):
    """One process of the parallel oracle sample: network b of the sweep,
    rebuilt alone (same graph and Philox keys as inside the batch) and
    stepped from step 0.  With target_s, a 200-step calibration run sets
    the step count to about target_s seconds (at most `steps`)."""
    try:
        import oracle
        inst = si.batched_sweep_params(n_nets, base_seed)[b]
        p = si.problem(si.BRUNEL, [inst], delay=15, n_steps=min(200, steps), seed=base_seed, threads=1,
                       inst_index0=b)
        if target_s:
            t0 = time.monotonic()
            oracle.run(p, inst_key0=b)
            dt = time.monotonic() - t0
            p.n_steps = int(min(steps, max(200, 200 * target_s / max(dt, 1e-3))))
        else:
            p.n_steps = steps
        barrier.wait(timeout=900)
        t0 = time.monotonic()  # system-wide clock: comparable between the processes
        r = oracle.run(p, inst_key0=b)
        out.put((b, p.n_steps, int(r["events"]), t0, time.monotonic(), p.n_edges))
    except Exception as e:  # reported to the parent, which falls back to one process
        barrier.abort()
        out.put((b, -1, 0, 0.0, 0.0, repr(e)))


def oracle_parallel(name: str, rank: int, steps: int, target_s: float | None, timeout_s: float = 1800.0):
    """The oracle on the first networks of a batched sweep, one process per
    host core (as many as the free host memory holds, each network's graph
    in its generator and in the oracle), all started together behind a
    barrier.  Returns (events/s over the wall time of the slowest, cores,
    description) or None if a process failed."""
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
    barrier, out = ctx.Barrier(k), ctx.Queue()
    procs = [ctx.Process(target=_oracle_process, args=(base, n_nets, b, steps, target_s, barrier, out), daemon=True)
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
        why = [r[5] for r in res if r[1] < 0] or [f"{k - len(res)} of {k} processes did not report"]
        print(f"parallel oracle sample failed ({why[0]}); timing one process instead", file=sys.stderr)
        return None
    events = sum(r[2] for r in res)
    wall = max(r[4] for r in res) - min(r[3] for r in res)
    n_steps = sorted(r[1] for r in res)
    desc = (f"networks 0-{k - 1} of the sweep, one process each on {k} host cores "
            f"({sum(p.n for p in params[:k])} neurons, {sum(r[5] for r in res)} synapses), "
            + (f"{n_steps[0]}-{n_steps[-1]} steps from step 0 (set for about {target_s:.0f} s per process, "
               f"at most {steps})" if target_s
               else f"{n_steps[0]} steps from step 0"))
    return events / wall, k, desc, wall


def cpu_baseline(prob, steps: int, target_s: float = 15.0, name: str = "", rank: int = 0):
    import oracle
    if sweep_size(name):
        r = oracle_parallel(name, rank, steps, target_s)
        if r is not None:
            value, cores, desc, wall = r
            return {"value": value, "unit": "synaptic events/s", "cores": cores, "kind": "oracle",
                    "sample": desc + ", single-threaded C oracle per process", "seconds": round(wall, 3)}
    sub, desc = oracle_sample(prob)
    sub.n_steps = 200
    t0 = time.perf_counter()
    r = oracle.run(sub)
    dt = time.perf_counter() - t0
    if dt < target_s / 4:
        sub.n_steps = int(min(steps, 200 * target_s / max(dt, 1e-3)))
        t0 = time.perf_counter()
        r = oracle.run(sub)
        dt = time.perf_counter() - t0
    return {"value": r["events"] / dt, "unit": "synaptic events/s", "cores": 1, "kind": "oracle",
            "sample": f"{desc}, {sub.n_steps} steps from step 0, single-threaded C oracle",
            "seconds": round(dt, 3), "realtime_factor": sub.n_steps * DT_MS * 1e-3 / dt}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
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

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


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


def launch_bytes(net, prob, t0: int, n: int, edge_bytes: int) -> list:
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
        out.append(int(deg[ids[m]].sum()) * edge_bytes + int(m.sum()) * B_SPIKE_DELIVERED)
    return out


def step_bytes(prob, edge_bytes: int, events: int, delivered: int, emitted: int, steps: int) -> float:
    per_neuron = B_NEURON[prob.model] + (B_NEURON_STDP if prob.stdp else 0)
    return (events * edge_bytes + delivered * B_SPIKE_DELIVERED +
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


def run_ours(args, rank, world, dist):
    import torch
    import paper_1912_07423_b300 as snn

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", 0)))
    torch.cuda.set_device(dev)
    t_gen = time.perf_counter()
    prob = workload(args.workload, rank)
    t_gen = time.perf_counter() - t_gen
    hbm, peak_kind = peaks()
    cap = int(prob.n * (args.warmup + args.steps + args.profile_steps) * 0.05) + (1 << 20)

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

    # ---- headline: batched + int16, timed on the device
    recv_mode = {"auto": snn.RECV_AUTO, "global": snn.RECV_GLOBAL, "tiled": snn.RECV_TILED,
                 "bulk": snn.RECV_BULK}[args.receive]
    lazy = prob.stdp and args.plasticity == "lazy"
    net = snn.Network(prob, w16=True, receive=recv_mode, log_capacity=cap, lazy=lazy, lazy_fifo=args.lazy_fifo)
    info = net.info()
    recv_kind = info["receive"]
    net.step(args.warmup)
    net.sync()
    clocks = ClockSampler(dev.index)
    clocks.start()
    t_main, ev_main, sp_main = timed(net, args.steps)
    clk = clocks.stop()
    t_a = args.warmup
    deliv_main = delivered_spikes(net, prob, t_a, t_a + args.steps)
    # ---- per-kernel times (CUDA events around every kernel, same stream)
    n_prof = min(args.steps, args.profile_steps)
    t_p0 = t_a + args.steps
    c0 = net.counters()
    phases = net.step_profiled(n_prof)
    c1 = net.counters()
    bytes_each = launch_bytes(net, prob, t_p0, min(n_prof, 16), info["edge_bytes"])
    ev_p, sp_p = c1["events"] - c0["events"], c1["spikes"] - c0["spikes"]
    deliv_p = delivered_spikes(net, prob, t_p0, t_p0 + n_prof)
    mem = info["device_bytes"]
    net.close()
    del net
    torch.cuda.empty_cache()

    t_max = max_over_ranks(t_main)
    ev_total = sum_over_ranks(ev_main)
    value = ev_total / t_max
    recv_ms = phases["receive"] / n_prof
    recv_bytes = (ev_p * info["edge_bytes"] + deliv_p * B_SPIKE_DELIVERED) / n_prof
    achieved = recv_bytes / (recv_ms * 1e-3) / 1e9
    step_b = step_bytes(prob, info["edge_bytes"], ev_main, deliv_main, sp_main, args.steps)
    step_frac = (step_b / (hbm * 1e9)) / t_main

    out = {"metric": METRIC, "value": value, "unit": "synaptic events/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "int16 weights, int32 input, f32 state",
           "data": "synthetic (seeded graphs, no dataset)",
           "config": {"workload": args.workload, "networks": len(prob.instances), "neurons": prob.n,
                      "synapses": prob.n_edges, "delay_steps": prob.delay, "dt_ms": DT_MS,
                      "receive": recv_kind, "tiles": info["n_tiles"], "weights": "int16 x 2^shift(row)",
                      "edge_bytes": info["edge_bytes"],
                      "l2": "inputs larger than L2 (edge arrays %.1f GB >> 126 MB)" % (prob.n_edges * 6 / 1e9),
                      "parallelism": f"replicas x{world} (independent networks, no collective)",
                      "graph_gen_s": round(t_gen, 1), "device_bytes": mem,
                      **({"plasticity": ("lazy, history %d steps" % (args.lazy_fifo or 128)) if lazy else "eager"}
                         if prob.stdp else {})},
           "realtime_factor": args.steps * DT_MS * 1e-3 / t_max,
           "spikes": int(sp_main), "events": int(ev_main),
           "roofline": {"kernel": f"k_receive_{recv_kind}", "bound": "hbm", "achieved": achieved, "peak": hbm,
                        "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": (traffic_ratio() * recv_bytes if traffic_ratio() and recv_kind == "tiled" else None),
                        "launch_ms": recv_ms,
                        "bytes_per_launch": recv_bytes, "launches": n_prof,
                        "bytes_each": bytes_each[:16],
                        # effective bytes per delivered event (edges + per-spike records) and the
                        # events/s the measured HBM rate allows for the edges alone
                        "bytes_per_event": recv_bytes * n_prof / max(ev_p, 1),
                        "edge_only_ceiling_events_per_s": hbm * 1e9 / info["edge_bytes"]},
           "step_roofline": {"bytes_per_step": step_b / args.steps, "frac": step_frac, "peak": hbm,
                             "unit": "GB/s", "achieved": step_b / t_main / 1e9,
                             "bytes_per_event": step_b / max(ev_main, 1)},
           "phase_ms_per_step": {k: v / n_prof for k, v in phases.items()},
           "gpu_launches": gpu_launches(args.steps, recv_kind, prob.stdp, lazy),
           "clocks": clk}

    # ---- plain single-precision weights + global-atomic receive, same networks
    if not args.no_plain:
        net = snn.Network(prob, w16=False, receive=snn.RECV_GLOBAL, log_capacity=cap, lazy=lazy,
                          lazy_fifo=args.lazy_fifo)
        net.step(args.warmup)
        net.sync()
        t_pl, ev_pl, sp_pl = timed(net, args.steps)
        net.close()
        del net
        torch.cuda.empty_cache()
        out["plain_fp32"] = {"value": sum_over_ranks(ev_pl) / max_over_ranks(t_pl), "unit": "synaptic events/s",
                             "receive": "global", "weights": "binary32",
                             "ms_per_step": t_pl * 1e3 / args.steps,
                             "realtime_factor": args.steps * DT_MS * 1e-3 / t_pl}
        out["speedup_vs_plain_fp32"] = out["value"] / out["plain_fp32"]["value"]

    # ---- the same networks through the generic update (Section III-B): Brunel
    # written as a specialisation of the LIF building block
    if not args.no_generic and prob.model == si.BRUNEL and not prob.stdp:
        gprob = dataclasses.replace(prob, model=snn.MODEL_BRUNEL_LIF)
        net = snn.Network(gprob, w16=True, receive=recv_mode, log_capacity=cap)
        net.step(args.warmup)
        net.sync()
        t_g, ev_g, sp_g = timed(net, args.steps)
        net.close()
        del net
        torch.cuda.empty_cache()
        out["generic_update"] = {"value": sum_over_ranks(ev_g) / max_over_ranks(t_g), "unit": "synaptic events/s",
                                 "ms_per_step": t_g * 1e3 / args.steps,
                                 "model": "Brunel from the LIF building block (SNN_MODEL_BRUNEL_LIF)",
                                 "same_events_and_spikes": bool(ev_g == ev_main and sp_g == sp_main)}

    # ---- end to end through the C ABI from host buffers
    if not args.no_e2e:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        net = snn.Network(prob, w16=True, receive=recv_mode, log_capacity=cap, lazy=lazy,
                          lazy_fifo=args.lazy_fifo)  # h2d of the graph
        t1 = time.perf_counter()
        net.step(args.steps)
        net.sync()
        t2 = time.perf_counter()
        steps_h, ids_h = net.spikes()  # d2h of the raster
        t_e2e = time.perf_counter() - t0
        parts = {"create_and_build_s": t1 - t0, "steps_s": t2 - t1, "raster_readout_s": t0 + t_e2e - t2}
        c = net.counters()
        net.close()
        del net
        torch.cuda.empty_cache()
        h2d = prob.row_off.nbytes + prob.tgt.nbytes + prob.w.nbytes
        d2h = 8 * int(c["spikes"])
        out["e2e"] = {"value": sum_over_ranks(c["events"]) / max_over_ranks(t_e2e), "unit": "synaptic events/s",
                      "seconds": t_e2e, "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                      "includes": "snn_create + snn_build_graph from host arrays + snn_step(K) + snn_read_spikes",
                      "parts": parts}

    # ---- adjacency construction on the GPU (Fig. 2) for the same networks
    if not args.no_graph:
        out["graph_construction"] = graph_construction(prob, dev, hbm)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:  # the baseline is a one-GPU figure
        out["cpu_baseline"] = cpu_baseline(prob, args.steps, name=args.workload, rank=rank)
    return out


def run_reference(args, rank):
    """The oracle, as it stands, on a bounded sample of the same workload,
    on the host cores."""
    import oracle
    # the run starts at step 0, where the delay FIFO delivers nothing for d
    # steps: at least 100 steps, so that a short run still measures events
    n_steps = max(args.warmup + args.steps, 100)
    r = oracle_parallel(args.workload, rank, n_steps, None) if sweep_size(args.workload) else None
    if r is not None:
        value, cores, desc, dt = r
    else:
        prob = workload(args.workload, rank)
        sub, desc = oracle_sample(prob)
        sub.n_steps = n_steps
        t0 = time.perf_counter()
        res = oracle.run(sub)
        dt = time.perf_counter() - t0
        value, cores = res["events"] / dt, 1
        desc = f"{desc}, {n_steps} steps"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "synaptic events/s", "n_gpus": 0,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / n_steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 state, int32 input",
            "data": "synthetic (seeded graphs, no dataset)",
            "config": {"workload": args.workload, "sample": desc},
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
    ap.add_argument("--profile-steps", type=int, default=500)
    ap.add_argument("--receive", choices=["auto", "global", "tiled", "bulk"], default="auto")
    ap.add_argument("--plasticity", choices=["eager", "lazy"], default="eager",
                    help="Update Synapses form for plastic workloads (brunel_stdp_100k; eager measured faster)")
    ap.add_argument("--lazy-fifo", type=int, default=0, help="lazy plasticity: history length (0: 128)")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-generic", action="store_true", help="skip timing the generic-update model")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-graph", action="store_true", help="skip timing the GPU adjacency construction")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
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
