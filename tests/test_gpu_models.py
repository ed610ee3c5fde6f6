"""Models of the generic update (Section III-B) through the C ABI.

SNN_MODEL_BRUNEL_LIF is Brunel written as a specialisation of the LIF
building block: the generic kernel must reproduce the fixed Brunel oracle
bit for bit.  SNN_MODEL_RELAY is the paper's tutorial model, compared with
the oracle's definition of it.
"""
import dataclasses

import numpy as np
import pytest

import oracle
import snn_inputs as si
from test_gpu_parity import RECV, oracle_run
from test_oracle_pins import _relay_problem

pytestmark = pytest.mark.gpu

MODEL_RELAY, MODEL_BRUNEL_LIF = 2, 3


def run_model(snn, prob, model, n_steps=None, receive="tiled", chunk=None):
    n_steps = prob.n_steps if n_steps is None else n_steps
    g = dataclasses.replace(prob, model=model)
    net = snn.Network(g, receive=RECV[receive], log_capacity=prob.n * max(n_steps, 1) + 4096)
    try:
        assert net.info()["model_state_bytes"] == snn.MODEL_STATE_DTYPE[model].itemsize
        t = 0
        while t < n_steps:
            k = n_steps - t if chunk is None else min(chunk, n_steps - t)
            net.step(k)
            t += k
        net.sync()
        steps, ids = net.spikes()
        return {"steps": steps, "ids": ids, "state": net.read("model"), "acc0": net.read("acc0"),
                "counters": net.counters()}
    finally:
        net.close()


def assert_brunel_parity(g, o):
    assert np.array_equal(g["steps"], o["steps"]) and np.array_equal(g["ids"], o["ids"])
    assert np.array_equal(g["state"]["V"].view(np.uint32), np.asarray(o["V"], np.float32).view(np.uint32))
    assert np.array_equal(g["state"]["r"].astype(np.int32), np.asarray(o["r"], np.int32))
    assert np.array_equal(g["acc0"], np.asarray(o["acc0"], np.int32))
    assert g["counters"]["events"] == o["events"]
    assert g["counters"]["spikes"] == len(o["ids"])


@pytest.mark.parametrize("receive", ["global", "tiled", "bulk"])
def test_brunel_lif_equals_brunel_oracle(gpu, receive):
    """Brunel 12.5k, 15-step delay, 2,000 steps, through the generic update."""
    prob = si.brunel_12k5(seed=1, n_steps=2000)
    o = oracle.run(prob)
    assert len(o["ids"]) > 10000
    assert_brunel_parity(run_model(gpu, prob, MODEL_BRUNEL_LIF, receive=receive, chunk=700), o)


def test_brunel_lif_uneven_batch(gpu):
    """Uneven networks of the sweep recipe (ragged instance sizes)."""
    prob = si.batched_sweep(n_nets=5, base_seed=11, n_steps=400, n_lo=300, n_hi=4000)
    o = oracle.run(prob)
    assert_brunel_parity(run_model(gpu, prob, MODEL_BRUNEL_LIF), o)


@pytest.mark.parametrize("d", [1, 2, 5])
@pytest.mark.parametrize("receive", ["global", "tiled"])
def test_relay_tutorial_model(gpu, d, receive):
    """Listing 1: two populations of 100 taking turns exciting each other."""
    prob, _ = _relay_problem(100, 100, 0.05, d, 60, seed=3)
    prob.instances[0].n_exc = 100
    prob.model = MODEL_RELAY
    o = oracle.relay_raster(prob)
    g = run_model(gpu, prob, MODEL_RELAY, receive=receive)
    assert len(o["ids"]) > 500
    assert np.array_equal(g["steps"], o["steps"]) and np.array_equal(g["ids"], o["ids"])
    assert np.array_equal(g["acc0"].astype(np.int64), o["acc0"])
    assert g["counters"]["events"] == o["events"]
    assert not g["state"]["flag"].any()  # every flag clears at the first update


def test_relay_model_on_ragged_instances(gpu):
    """The relay model on three Brunel-shaped graphs of ragged sizes (inhibitory
    weights included: a neuron fires when its summed input is nonzero)."""
    insts = [si.brunel_instance(n, k=k, graph_seed=20 + i) for i, (n, k) in enumerate([(257, 6), (1000, 5), (31, 3)])]
    for inst in insts:
        inst.n_exc = inst.n // 10  # the active first population
    prob = si.problem(si.BRUNEL, insts, delay=2, n_steps=50, seed=5)
    prob.model = MODEL_RELAY
    o = oracle.relay_raster(prob)
    g = run_model(gpu, prob, MODEL_RELAY)
    assert len(o["ids"]) > 100
    assert np.array_equal(g["steps"], o["steps"]) and np.array_equal(g["ids"], o["ids"])
    assert g["counters"]["events"] == o["events"]


def test_model_state_write_is_read_back(gpu):
    """SNN_FIELD_MODEL round-trips, and a written state is the one the next
    update starts from (a silenced network stays silent)."""
    prob, _ = _relay_problem(100, 100, 0.05, 1, 10, seed=3)
    prob.instances[0].n_exc = 100
    g = dataclasses.replace(prob, model=MODEL_RELAY)
    net = gpu.Network(g, receive=RECV["tiled"], log_capacity=1 << 16)
    try:
        st = net.read("model")
        assert st["flag"][:100].all() and not st["flag"][100:].any()
        st["flag"][:] = 0
        net.write("model", st)
        assert not net.read("model")["flag"].any()
        net.step(10)
        net.sync()
        assert len(net.spikes()[1]) == 0
    finally:
        net.close()


def test_large_raster_readout(gpu):
    """A raster larger than the readout's chunked host copy (150M spikes, 600 MB
    per array): the tutorial model on a ring of 1M neurons that all start active
    fires every neuron at every step."""
    n, T = 1_000_000, 150
    inst = si.brunel_instance(n, k=0)
    inst.n_exc = n
    prob = si.Problem(model=MODEL_RELAY, instances=[inst], delay=1, seed=1, n_steps=T,
                      inst_off=np.array([0, n], np.uint32), row_off=np.arange(n + 1, dtype=np.uint64),
                      tgt=((np.arange(n, dtype=np.uint64) + 1) % n).astype(np.uint32), w=np.full(n, 5, np.int32))
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=n * T)
    try:
        net.step(T)
        net.sync()
        steps, ids = net.spikes()
        assert len(ids) == n * T
        assert (steps.reshape(T, n) == np.arange(T, dtype=np.uint32)[:, None]).all()
        assert (ids.reshape(T, n) == np.arange(n, dtype=np.uint32)[None, :]).all()
        assert net.counters()["events"] == n * T
    finally:
        net.close()
