"""Lazy Update Synapses (Section III-A-1) against the eager oracle.

The lazy form leaves the plastic synapses of a row stale until the row
transmits a spike or its history of F steps would otherwise run out, then
replays the missed steps in one pass.  The paper states that this reaches
the eager rule's result; here every weight, trace, spike and pending input
must equal the oracle's (which applies the rule eagerly, every step) bit for
bit, whatever F, the delay, the weight storage or the receive form.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import snn_inputs as si
from test_gpu_parity import RECV, _fields, assert_parity, oracle_run

pytestmark = pytest.mark.gpu


def run_lazy(snn, prob, n_steps=None, *, fifo=0, w16=True, receive="tiled", reads=(), identity_writes=()):
    """Simulate with lazy plasticity.  reads: steps after which W and x are
    read (each read brings every row up to date first; the copies are
    returned); identity_writes: steps after which W and x are written back
    unchanged (a flush, then a write)."""
    n_steps = prob.n_steps if n_steps is None else n_steps
    net = snn.Network(prob, w16=w16, receive=RECV[receive], log_capacity=prob.n * max(n_steps, 1) + 4096,
                      lazy=True, lazy_fifo=fifo)
    try:
        cuts = sorted(set(reads) | set(identity_writes) | {n_steps})
        t, seen = 0, {}
        for c in cuts:
            if c > t:
                net.step(c - t)
                t = c
            if c in reads:
                seen[c] = {"w": net.read("w"), "x": net.read("x"), "y": net.read("y")}
            if c in identity_writes:
                net.write("w", net.read("w"))
                net.write("x", net.read("x"))
        net.sync()
        out = {f: net.read(f) for f in _fields(prob)}
        out["steps"], out["ids"] = net.spikes()
        out["counters"] = net.counters()
        out["seen"] = seen
        return out
    finally:
        net.close()


def small_stdp(n_steps=3000):
    return si.brunel_stdp_100k(seed=2, n_steps=n_steps, n=4000, k=400)


@pytest.mark.parametrize("fifo", [0, 2, 17, 50, 63, 64, 65, 127])
@pytest.mark.parametrize("receive", ["global", "tiled"])
def test_lazy_equals_eager_oracle(gpu, fifo, receive):
    """Brunel+ at 4,000 neurons (in-degree 400), 15-step delay, 3,000 steps:
    the default history (128 steps, the most the two history words hold),
    the shortest (every row replayed every other step), an odd length, the
    paper's 50, the lengths around the boundary of the two words and one
    step below the longest."""
    prob = small_stdp()
    o = oracle_run("bstdp4k", prob)
    g = run_lazy(gpu, prob, fifo=fifo, receive=receive)
    assert len(o["ids"]) > 1000
    assert not np.array_equal(o["w"], prob.w)  # plasticity did something
    assert_parity(g, o, prob)


def test_lazy_binary32_weights(gpu):
    prob = small_stdp()
    o = oracle_run("bstdp4k", prob)
    assert_parity(run_lazy(gpu, prob, w16=False, receive="global"), o, prob)


def test_lazy_with_the_bulk_receive(gpu):
    prob = small_stdp(n_steps=1500)
    o = oracle.run(prob)
    assert_parity(run_lazy(gpu, prob, fifo=40, receive="bulk"), o, prob)


@pytest.mark.parametrize("fifo", [2, 50])
def test_lazy_delay_one(gpu, fifo):
    """d = 1: a row transmits at the step its neuron spikes, and the
    arrival is the next step."""
    prob = si.brunel_stdp_100k(seed=4, n_steps=800, n=1500, k=150)
    prob.delay = 1
    o = oracle.run(prob)
    assert_parity(run_lazy(gpu, prob, fifo=fifo), o, prob)


@pytest.mark.parametrize("delay", [2, 40])
def test_lazy_delays(gpu, delay):
    """Delays below and at the order of the history length."""
    prob = si.brunel_stdp_100k(seed=6, n_steps=900, n=2500, k=250)
    prob.delay = delay
    o = oracle.run(prob)
    assert_parity(run_lazy(gpu, prob, fifo=20), o, prob)


def test_reads_mid_run_are_the_eager_state(gpu):
    """Reading W or x between steps brings every stale row up to date: the
    values equal the eager oracle's after that many steps, and the run goes
    on unchanged afterwards."""
    prob = small_stdp(n_steps=1200)
    cuts = (1, 333, 777)
    g = run_lazy(gpu, prob, fifo=50, reads=cuts)
    for c in cuts:
        oc = oracle.run(dataclasses.replace(prob, n_steps=c))
        for f in ("w", "x", "y"):
            a = np.asarray(g["seen"][c][f])
            b = np.asarray(oc[f])
            if a.dtype == np.float32:
                a, b = a.view(np.uint32), b.astype(np.float32).view(np.uint32)
            assert np.array_equal(a, b), f"{f} after {c} steps differs at {np.flatnonzero(a != b)[:8]}"
    assert_parity(g, oracle.run(prob), prob)


def test_identity_writes_mid_run(gpu):
    """Writing W and x back unchanged between steps (a flush, then the
    write) leaves the run equal to the oracle's."""
    prob = small_stdp(n_steps=1000)
    o = oracle.run(prob)
    assert_parity(run_lazy(gpu, prob, fifo=30, identity_writes=(10, 499, 500, 901)), o, prob)


def test_lazy_uneven_batch(gpu):
    """Three plastic networks of different sizes in one context (the replay
    finds each row's instance, excitatory count and constants)."""
    insts = [si.brunel_instance(n, k=k, graph_seed=10 + i, stdp=True)
             for i, (n, k) in enumerate([(1000, 100), (3001, 300), (2222, 222)])]
    prob = si.problem(si.BRUNEL, insts, delay=15, n_steps=1000, seed=3, stdp=True)
    o = oracle.run(prob)
    assert_parity(run_lazy(gpu, prob, fifo=50), o, prob)


def test_lazy_reset_repeats_the_run(gpu):
    prob = si.brunel_stdp_100k(seed=5, n_steps=600, n=2000, k=200)
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=1 << 20, lazy=True)
    net.step(600)
    a = net.spikes()
    wa = net.read("w")
    net.reset()
    net.step(600)
    b = net.spikes()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(wa, net.read("w"))
    net.close()
