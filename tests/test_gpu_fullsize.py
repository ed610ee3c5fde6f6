"""Parity at the full workload sizes and run lengths, in the launch
configuration bench.py times (default receive, 16-bit weights, CUDA-graph
steps, the fused step where it applies).

The batched sweep of 256 networks is too large for the oracle to run whole,
but its networks are independent and each one's random draws depend only on
(seed, instance, neuron, step): sampled networks are re-run alone by the
oracle, for all 5,000 steps, and must match bit for bit.  The 1M-neuron
Vogels network (1,000 steps) and the 100k-neuron Brunel+ network (10,000
steps, raster, potentials and weights at the end) are compared whole.  The
oracle runs take minutes, so they start together in host processes when the
module's first test asks for them, while the GPU runs the other tests.
"""
import concurrent.futures as cf
import dataclasses
import functools
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import snn_inputs as si
from test_gpu_parity import assert_tuned_fastest

pytestmark = pytest.mark.gpu

SWEEP_STEPS, V1M_STEPS, STDP_STEPS = 5000, 1000, 10000


def _sweep_sample(sizes) -> list:
    """Networks of the sweep re-run alone: the smallest, the largest and
    random ones (8 in all)."""
    rng = np.random.default_rng(11)
    pick = {int(np.argmin(sizes)), int(np.argmax(sizes))}
    while len(pick) < 8:
        pick.add(int(rng.integers(0, len(sizes))))
    return sorted(pick)


def _oracle_job(kind: str, arg: int):
    """One oracle run in a host process (its own graph, built from the seeds)."""
    import oracle as orc
    import snn_inputs as sin
    if kind == "sweep":
        params = sin.batched_sweep_params(256, 1)
        p = sin.problem(sin.BRUNEL, [params[arg]], delay=15, n_steps=SWEEP_STEPS, seed=1, threads=1, inst_index0=arg)
        o = orc.run(p, inst_key0=arg)
        return {k: o[k] for k in ("steps", "ids", "V", "events")}
    if kind == "v1m":
        o = orc.run(sin.vogels_1m(seed=1, n_steps=V1M_STEPS))
        return {k: o[k] for k in ("steps", "ids", "V", "events")}
    if kind == "stdp":
        o = orc.run(sin.brunel_stdp_100k(seed=1, n_steps=STDP_STEPS))
        return {k: o[k] for k in ("steps", "ids", "V", "w", "events")}
    raise ValueError(kind)


@pytest.fixture(scope="module")
def oracle_runs():
    """Futures of every oracle run this module compares with."""
    sizes = np.array([inst.n for inst in si.batched_sweep_params(256, 1)])
    jobs = [("stdp", 0), ("v1m", 0)] + [("sweep", b) for b in _sweep_sample(sizes)]
    ex = cf.ProcessPoolExecutor(max_workers=max(1, min(len(jobs), len(os.sched_getaffinity(0)))),
                                mp_context=mp.get_context("spawn"))
    futs = {job: ex.submit(_oracle_job, *job) for job in jobs}
    yield futs
    ex.shutdown(wait=True, cancel_futures=True)


def _gpu_run(gpu, prob, steps, chunks=(100,), **kw):
    net = gpu.Network(prob, log_capacity=prob.n * steps // 5 + (1 << 20), **kw)
    t = 0
    for c in chunks:
        net.step(c)
        t += c
    if t < steps:
        net.step(steps - t)
    net.sync()
    V = net.read("model")["V"] if prob.model == gpu.MODEL_BRUNEL_LIF else net.read("V")
    out = {"steps_ids": net.spikes(), "V": V, "info": net.info(), "counters": net.counters()}
    if prob.stdp:
        out["w"] = net.read("w")
    net.close()
    return out


@functools.lru_cache(maxsize=1)
def _sweep():
    return si.batched_sweep(256, base_seed=1, n_steps=0)


def test_batched_sweep_256_sampled_networks_whole_run(gpu, oracle_runs):
    """The fixed Brunel kernel (fused step) over the whole 5,000-step run:
    8 sampled networks re-run alone by the oracle, raster and final V."""
    prob = _sweep()
    g = _gpu_run(gpu, prob, SWEEP_STEPS, chunks=(100, 200, 1000))
    assert_tuned_fastest(g["info"])
    gs, gi = g["steps_ids"]
    sizes = np.array([inst.n for inst in prob.instances])
    for b in _sweep_sample(sizes):
        o = oracle_runs[("sweep", b)].result()
        lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
        m = (gi >= lo) & (gi < hi)
        assert len(o["ids"]) > 0
        assert np.array_equal(gs[m], o["steps"]), b
        assert np.array_equal(gi[m] - lo, o["ids"]), b
        assert np.array_equal(g["V"][lo:hi].view(np.uint32), o["V"].view(np.uint32)), b


def test_batched_sweep_256_generic_update(gpu):
    """Brunel from the LIF building block through the generic update (bench.py's
    generic_update line), 400 steps, sampled networks re-run alone."""
    prob = _sweep()
    steps = 400
    run = dataclasses.replace(prob, model=gpu.MODEL_BRUNEL_LIF)
    g = _gpu_run(gpu, run, steps, chunks=(100, 200))
    assert_tuned_fastest(g["info"])
    gs, gi = g["steps_ids"]
    sizes = np.array([inst.n for inst in prob.instances])
    for b in sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 37, 200}):
        sub = si.sub_problem(prob, b, n_steps=steps)
        o = oracle.run(sub, inst_key0=b)
        lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
        m = (gi >= lo) & (gi < hi)
        assert len(o["ids"]) > 0
        assert np.array_equal(gs[m], o["steps"]), b
        assert np.array_equal(gi[m] - lo, o["ids"]), b
        assert np.array_equal(g["V"][lo:hi].view(np.uint32), o["V"].view(np.uint32)), b


def test_vogels_1m_whole_run(gpu, oracle_runs):
    """Vogels-Abbott 1M neurons, in-degree 1,000, all 1,000 steps, through the
    global receive with row weights (4 bytes per event)."""
    prob = si.vogels_1m(seed=1, n_steps=V1M_STEPS)
    g = _gpu_run(gpu, prob, V1M_STEPS)
    assert_tuned_fastest(g["info"])
    if g["info"]["receive"] == "global":
        assert g["info"]["edge_bytes"] == 4
    del prob
    o = oracle_runs[("v1m", 0)].result()
    gs, gi = g["steps_ids"]
    assert len(o["ids"]) > 1000
    assert np.array_equal(gs, o["steps"]) and np.array_equal(gi, o["ids"])
    assert np.array_equal(g["V"].view(np.uint32), o["V"].view(np.uint32))
    assert g["counters"]["events"] == o["events"]


@pytest.mark.parametrize("lazy", [False, True])
def test_brunel_stdp_100k_whole_run(gpu, oracle_runs, lazy):
    """Brunel+ 100k, all 10,000 steps: eager Update Synapses, and the lazy form
    bench.py times (128-step history); raster, final V and weights."""
    prob = si.brunel_stdp_100k(seed=1, n_steps=STDP_STEPS)
    g = _gpu_run(gpu, prob, STDP_STEPS, chunks=(100, 2000), lazy=lazy)
    assert_tuned_fastest(g["info"])
    o = oracle_runs[("stdp", 0)].result()
    gs, gi = g["steps_ids"]
    assert len(o["ids"]) > 1000
    assert np.array_equal(gs, o["steps"]) and np.array_equal(gi, o["ids"])
    assert np.array_equal(g["V"].view(np.uint32), o["V"].view(np.uint32))
    assert np.array_equal(g["w"], o["w"])
    assert not np.array_equal(o["w"], prob.w)
    assert g["counters"]["events"] == o["events"]


def test_sweep_adjacency_construction_sampled_jobs(gpu):
    """snn_expand_jobs (Fig. 2) on the sweep's full job list, as bench.py times
    it (one job per neuron: its out-degree of values from its own instance,
    2.9e9 values), checked job by job against the oracle on a sample: the
    shortest and longest jobs, the first and last, and random ones."""
    import torch
    prob = _sweep()
    deg = np.diff(prob.row_off.astype(np.int64)).astype(np.uint32)
    inst_of = np.repeat(np.arange(len(prob.instances)), np.diff(prob.inst_off.astype(np.int64)))
    jobs = np.zeros(prob.n, dtype=gpu.JOB_DTYPE)
    jobs["n"] = deg
    jobs["a"] = prob.inst_off[inst_of]
    jobs["b"] = prob.inst_off[inst_of + 1]
    jobs["o"] = prob.row_off[:-1]
    E = int(prob.row_off[-1])
    out = torch.empty(E, dtype=torch.int32, device="cuda")
    gpu.expand_jobs(torch.from_numpy(jobs.view(np.uint8)).cuda(), 1, E, out=out)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    sample = {0, prob.n - 1, int(np.argmin(deg)), int(np.argmax(deg))} | set(rng.integers(0, prob.n, 60).tolist())
    ojobs = jobs.view(oracle.JOB_DTYPE)
    for j in sorted(sample):
        lo, n = int(jobs["o"][j]), int(jobs["n"][j])
        got = out[lo:lo + n].cpu().numpy().view(np.uint32)
        assert np.array_equal(got, oracle.expand_job(ojobs[j], j, 1)), j
    del out
    torch.cuda.empty_cache()
