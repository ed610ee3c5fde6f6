"""Parity at the full workload sizes, in the launch configuration bench.py
times (default receive, 16-bit weights, CUDA-graph steps, re-planned tiles).

The batched sweep of 256 networks is too large for the oracle to run whole,
but its networks are independent and each one's random draws depend only on
(seed, instance, neuron, step): sampled networks are re-run alone by the
oracle and must match bit for bit.  The 1M-neuron Vogels network and the
100k-neuron Brunel+ network are compared whole over a window of steps.
"""
import dataclasses
import functools

import numpy as np
import pytest

import oracle
import snn_inputs as si

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("model", ["fixed", "generic"])
def test_batched_sweep_256_sampled_networks(gpu, model):
    """model: the fixed Brunel kernel, or Brunel from the LIF building block
    through the generic update (bench.py's generic_update line)."""
    prob = _sweep()
    steps = 400  # crosses the first re-plan of the work items (step 256)
    run = prob if model == "fixed" else dataclasses.replace(prob, model=gpu.MODEL_BRUNEL_LIF)
    g = _gpu_run(gpu, run, steps, chunks=(100, 200))
    assert g["info"]["receive"] == "tiled"
    gs, gi = g["steps_ids"]
    sizes = np.array([inst.n for inst in prob.instances])
    sample = sorted({int(np.argmin(sizes)), int(np.argmax(sizes)), 37, 200})
    for b in sample:
        sub = si.sub_problem(prob, b, n_steps=steps)
        o = oracle.run(sub, inst_key0=b)
        lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
        m = (gi >= lo) & (gi < hi)
        assert len(o["ids"]) > 0
        assert np.array_equal(gs[m], o["steps"]), b
        assert np.array_equal(gi[m] - lo, o["ids"]), b
        assert np.array_equal(g["V"][lo:hi].view(np.uint32), o["V"].view(np.uint32)), b


def test_vogels_1m_whole_network(gpu):
    prob = si.vogels_1m(seed=1, n_steps=120)
    g = _gpu_run(gpu, prob, 120)
    o = oracle.run(prob)
    gs, gi = g["steps_ids"]
    assert len(o["ids"]) > 1000
    assert np.array_equal(gs, o["steps"]) and np.array_equal(gi, o["ids"])
    assert np.array_equal(g["V"].view(np.uint32), o["V"].view(np.uint32))
    assert g["counters"]["events"] == o["events"]


@functools.lru_cache(maxsize=1)
def _stdp_100k():
    prob = si.brunel_stdp_100k(seed=1, n_steps=300)
    return prob, oracle.run(prob)


@pytest.mark.parametrize("lazy", [False, True])
def test_brunel_stdp_100k_whole_network(gpu, lazy):
    """Eager Update Synapses, and the lazy form bench.py times (128-step history)."""
    prob, o = _stdp_100k()
    g = _gpu_run(gpu, prob, 300, lazy=lazy)
    gs, gi = g["steps_ids"]
    assert len(o["ids"]) > 1000
    assert np.array_equal(gs, o["steps"]) and np.array_equal(gi, o["ids"])
    assert np.array_equal(g["V"].view(np.uint32), o["V"].view(np.uint32))
    assert np.array_equal(g["w"], o["w"])
    assert not np.array_equal(o["w"], prob.w)


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
