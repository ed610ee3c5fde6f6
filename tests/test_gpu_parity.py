"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Rasters, neuron state, pending input and (with STDP) weights must agree bit
for bit: the update is the same binary32 op sequence on both sides, input
is integer, and the random draws come from the same counter-based
generator implemented independently on each side.
"""
import numpy as np
import pytest

import oracle
import snn_inputs as si

pytestmark = pytest.mark.gpu

RECV = {"global": 1, "tiled": 2, "bulk": 3, "tiled_serial": 2, "persistent": 4}
# "tiled_serial": the tiled receive as its own kernel after the update even
# where the library would run both in one kernel per step (SNN_F_SERIAL)


def _fields(prob):
    f = ["V", "r", "acc0"]
    if prob.model == si.VOGELS:
        f += ["ge", "gi", "acc1"]
    if prob.stdp:
        f += ["x", "y", "w"]
    return f


def run_gpu(snn, prob, n_steps=None, *, w16=True, receive="global", overrides=(), state=None, chunk=None,
            packed=True):
    """Simulate through the C ABI; overrides (step, id, V) are written
    between steps, before that step's update, like the oracle applies them."""
    n_steps = prob.n_steps if n_steps is None else n_steps
    total = prob.n * max(n_steps, 1)
    cap = total + 4096 if total < 10_000_000 else total // 10 + 4096
    net = snn.Network(prob, w16=w16, receive=RECV[receive], log_capacity=cap, packed=packed,
                      serial=receive == "tiled_serial")
    fused_expected = (receive == "tiled" and w16 and prob.model == si.BRUNEL and not prob.stdp
                      and prob.delay >= 3)
    assert net.info()["fused"] == fused_expected
    try:
        if state:
            for k, v in state.items():
                net.write(k, v)
        t = 0
        for (ts, i, v) in sorted(overrides):
            if ts > t:
                net.step(ts - t)
                t = ts
            V = net.read("V")
            V[i] = v
            net.write("V", V)
        while t < n_steps:
            k = n_steps - t if chunk is None else min(chunk, n_steps - t)
            net.step(k)
            t += k
        net.sync()
        steps, ids = net.spikes()
        out = {f: net.read(f) for f in _fields(prob)}
        out.update(steps=steps, ids=ids, counters=net.counters())
        return out
    finally:
        net.close()


def assert_parity(g, o, prob):
    assert len(g["ids"]) == len(o["ids"]), (len(g["ids"]), len(o["ids"]))
    assert np.array_equal(g["steps"], o["steps"])
    assert np.array_equal(g["ids"], o["ids"])
    for f in _fields(prob):
        a, b = np.asarray(g[f]), np.asarray(o[f])
        if a.dtype == np.float32:
            a, b = a.view(np.uint32), b.astype(np.float32).view(np.uint32)
        assert np.array_equal(a, b), f"field {f} differs at {np.flatnonzero(a != b)[:8]}"
    assert g["counters"]["events"] == o["events"]
    assert g["counters"]["spikes"] == len(o["ids"])


_cache = {}


def oracle_run(key, prob, **kw):
    if key not in _cache:
        _cache[key] = oracle.run(prob, **kw)
    return _cache[key]


# ------------------------------------------------------------------ the configs
@pytest.mark.parametrize("w16", [True, False])
@pytest.mark.parametrize("receive", ["global", "tiled", "bulk", "persistent"])
def test_vogels_4k_full(gpu, w16, receive):
    """Vogels-Abbott, 4,000 neurons, 2 % connectivity, 1,000 steps."""
    prob = si.vogels_4k(seed=1, n_steps=1000)
    o = oracle_run("v4k", prob)
    g = run_gpu(gpu, prob, w16=w16, receive=receive)
    assert len(o["ids"]) > 1000
    assert_parity(g, o, prob)


@pytest.mark.parametrize("receive", ["global", "tiled", "bulk", "tiled_serial", "persistent"])
def test_brunel_12k5_full(gpu, receive):
    """Brunel, 12,500 neurons, C_E 1,000 / C_I 250, 15-step delay, 10,000 steps."""
    prob = si.brunel_12k5(seed=1, n_steps=10000)
    o = oracle_run("b12k5", prob)
    g = run_gpu(gpu, prob, w16=True, receive=receive)
    assert len(o["ids"]) > 100000
    assert_parity(g, o, prob)


@pytest.mark.parametrize("w16", [True, False])
@pytest.mark.parametrize("receive", ["global", "tiled", "bulk"])
def test_brunel_stdp_small(gpu, w16, receive):
    """Brunel+ at 4,000 neurons (in-degree 400), STDP, 15-step delay."""
    prob = si.brunel_stdp_100k(seed=2, n_steps=3000, n=4000, k=400)
    o = oracle_run("bstdp4k", prob)
    g = run_gpu(gpu, prob, w16=w16, receive=receive)
    assert len(o["ids"]) > 1000
    assert not np.array_equal(o["w"], prob.w)  # plasticity did something
    assert_parity(g, o, prob)


@pytest.mark.parametrize("receive", ["global", "tiled", "bulk", "tiled_serial", "persistent"])
def test_batched_uneven_parity(gpu, receive):
    """A batch of uneven Brunel networks in one context equals the oracle
    on the whole batch."""
    prob = si.batched_sweep(n_nets=12, base_seed=3, n_steps=1500, n_lo=37, n_hi=6000)
    o = oracle_run("batch12", prob)
    g = run_gpu(gpu, prob, receive=receive, chunk=700)
    assert_parity(g, o, prob)


def test_batched_instance_equals_alone(gpu):
    """Every instance of a batch behaves as if it ran alone (its Philox key
    is its instance index)."""
    prob = si.batched_sweep(n_nets=6, base_seed=5, n_steps=800, n_lo=300, n_hi=3000)
    g = run_gpu(gpu, prob, receive="tiled")
    for b in range(6):
        sub = si.sub_problem(prob, b)
        o = oracle.run(sub, inst_key0=b)
        lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
        m = (g["ids"] >= lo) & (g["ids"] < hi)
        assert np.array_equal(g["steps"][m], o["steps"])
        assert np.array_equal(g["ids"][m] - lo, o["ids"])


# ------------------------------------------------------------------ timing of the pipeline
@pytest.mark.parametrize("d", [1, 2, 15, 16])
@pytest.mark.parametrize("model", [si.VOGELS, si.BRUNEL])
def test_forced_spike_arrives_after_d_steps(gpu, d, model):
    """A spike forced at step tau reaches its targets' update at tau + d."""
    if model == si.VOGELS:
        inst = si.vogels_instance(300)
        w_e, w_i = 106168, -589824
    else:
        inst = si.brunel_instance(300, k=0)
        inst.lam = 0.0
        w_e, w_i = 6554, -32768
    inst.n_exc = 240
    edges = [(0, 5), (0, 77), (0, 299), (250, 5), (250, 6)]
    w = [w_e, w_e, w_e, w_i, w_i]
    prob = si.from_edges(model, inst, edges, w, delay=d, n_steps=40)
    ov = [(7, 0, 1000.0), (9, 250, 1000.0)]
    o = oracle.run(prob, overrides=ov)
    for receive in ("global", "tiled", "bulk", "tiled_serial", "persistent"):
        g = run_gpu(gpu, prob, overrides=ov, receive=receive)
        assert_parity(g, o, prob)


def test_largest_delay(gpu):
    """d = 1,000 steps, the largest delay the library takes (a ring of 1,000
    spike queues): a Brunel network driven to spike, 1,300 steps, every
    receive form."""
    prob = si.brunel_stdp_100k(seed=8, n_steps=1300, n=1200, k=120)
    prob.stdp = False
    prob.delay = 1000
    o = oracle.run(prob)
    assert int((o["steps"] >= 1000).sum()) > 100  # spikes after the first deliveries
    for receive in ("global", "tiled", "bulk", "tiled_serial", "persistent"):
        assert_parity(run_gpu(gpu, prob, receive=receive), o, prob)


@pytest.mark.parametrize("d", [1, 3])
def test_relay_network(gpu, d):
    """Listing 1's ping-pong network: S_{t+d} = out-neighbours(S_t)."""
    rng = np.random.Generator(np.random.PCG64(1))
    edges = [(j, i) for j in range(100) for i in range(100, 200) if rng.random() < 0.05]
    edges += [(j, i) for j in range(100, 200) for i in range(100) if rng.random() < 0.05]
    inst = si.brunel_instance(200, k=0)
    inst.n_exc, inst.tau_m, inst.v_th, inst.v_reset, inst.refractory_steps, inst.lam = 200, 1e-6, 0.05, 0.0, 0, 0.0
    prob = si.from_edges(si.BRUNEL, inst, edges, [6554] * len(edges), delay=d, n_steps=60)
    acc0 = np.zeros(200, np.int32)
    acc0[:100] = 6554
    state = {"V": np.zeros(200, np.float32), "acc0": acc0}
    ostate = {"V": np.zeros(200, np.float32), "ge": np.zeros(200, np.float32), "gi": np.zeros(200, np.float32),
              "r": np.zeros(200, np.int32), "x": np.zeros(200, np.float32), "y": np.zeros(200, np.float32),
              "acc0": acc0, "acc1": np.zeros(200, np.int32), "w": prob.w.copy()}
    o = oracle.run(prob, state=ostate)
    for receive in ("tiled", "bulk", "tiled_serial", "persistent"):
        g = run_gpu(gpu, prob, state=state, receive=receive)
        assert_parity(g, o, prob)
    assert len(o["ids"]) > 500
    assert_parity(g, o, prob)


# ------------------------------------------------------------------ edge cases
def test_empty_graph_and_ragged_instances(gpu):
    """No edges at all, instances of 1, 7, 255, 257 and 1000 neurons."""
    insts = [si.brunel_instance(n, k=0, nu_ratio=3.0) for n in (1, 7, 255, 257, 1000)]
    prob = si.problem(si.BRUNEL, insts, delay=2, n_steps=700, seed=9)
    assert prob.n_edges == 0
    o = oracle.run(prob)
    for receive in ("global", "tiled", "bulk", "persistent"):
        assert_parity(run_gpu(gpu, prob, receive=receive), o, prob)


def test_stdp_delay_one(gpu):
    prob = si.brunel_stdp_100k(seed=4, n_steps=800, n=1500, k=150)
    prob.delay = 1
    o = oracle.run(prob)
    assert_parity(run_gpu(gpu, prob, receive="tiled"), o, prob)


def test_unsorted_rows(gpu):
    """Rows need not be sorted: the global receive takes them; the tiled one
    refuses them with an argument error."""
    prob = si.brunel_12k5(seed=3, n_steps=300)
    rng = np.random.Generator(np.random.PCG64(0))
    tgt, w = prob.tgt.copy(), prob.w.copy()
    for j in range(0, prob.n, 97):
        a, b = int(prob.row_off[j]), int(prob.row_off[j + 1])
        p = rng.permutation(b - a)
        tgt[a:b], w[a:b] = tgt[a:b][p], w[a:b][p]
    prob.tgt, prob.w = tgt, w
    o = oracle.run(prob)
    assert_parity(run_gpu(gpu, prob, receive="global"), o, prob)
    with pytest.raises(gpu.SnnError) as ei:
        run_gpu(gpu, prob, receive="tiled")
    assert ei.value.status == -1


def test_invalid_graphs_are_rejected(gpu):
    base = si.brunel_12k5(seed=1, n_steps=10)
    # a target outside the source's instance
    two = si.batched_sweep(n_nets=2, base_seed=1, n_steps=10, n_lo=500, n_hi=600)
    bad = two.tgt.copy()
    bad[0] = int(two.inst_off[1]) + 3
    with pytest.raises(gpu.SnnError) as ei:
        gpu.Network(si.Problem(**{**two.__dict__, "tgt": bad}))
    assert ei.value.status == -1
    # a row whose weights are not one shift of int16 codes
    w = base.w.copy()
    w[int(base.row_off[5])] = 32769
    with pytest.raises(gpu.SnnError) as ei:
        gpu.Network(si.Problem(**{**base.__dict__, "w": w}), w16=True)
    assert ei.value.status == -1
    # the same weights are fine as binary32 lattice values
    gpu.Network(si.Problem(**{**base.__dict__, "w": w}), w16=False).close()


def test_log_overflow_is_reported(gpu):
    prob = si.brunel_12k5(seed=1, n_steps=400)
    net = gpu.Network(prob, log_capacity=1000)
    net.step(400)
    with pytest.raises(gpu.SnnError) as ei:
        net.sync()
    assert ei.value.status == -4
    net.log_clear()
    net.step(1)
    net.sync()
    net.close()


@pytest.mark.parametrize("name", ["vogels_4k", "brunel_stdp"])
def test_build_graph_rows_equals_per_synapse_weights(gpu, name):
    """snn_build_graph_rows (one weight per row, Table 2's population-typed
    synapses) loads the graph snn_build_graph loads from the same weights
    spread over the synapses: the weights read back, and the raster, V and
    (with STDP) the weights after a run are the same, and equal the oracle's."""
    if name == "vogels_4k":
        prob = si.vogels_4k(seed=4, n_steps=300)
    else:
        prob = si.brunel_stdp_100k(seed=2, n_steps=300, n=4000, k=400)
    o = oracle.run(prob)
    out = []
    for rows in (False, True):
        net = gpu.Network(prob, log_capacity=prob.n * 300, build_graph=False)
        try:
            if rows:
                net.build_graph_rows(prob.row_off, prob.tgt, prob.row_weights())
            else:
                net.build_graph(prob.row_off, prob.tgt, prob.w)
            w0 = net.read("w")
            net.step(300)
            steps, ids = net.spikes()
            out.append((w0, steps, ids, net.read("V"), net.read("w"), net.info()["edge_bytes"]))
        finally:
            net.close()
    (w0a, sa, ia, va, wa, ea), (w0b, sb, ib, vb, wb, eb) = out
    assert np.array_equal(w0a, prob.w) and np.array_equal(w0b, prob.w)
    assert np.array_equal(sa, sb) and np.array_equal(ia, ib) and ea == eb
    assert np.array_equal(va.view(np.uint32), vb.view(np.uint32)) and np.array_equal(wa, wb)
    assert np.array_equal(sb, o["steps"]) and np.array_equal(ib, o["ids"])
    assert np.array_equal(wb, o["w"])


def test_raster_log_regions(gpu):
    """The raster log keeps each instance's spikes in its own region, its
    share of log_capacity by neurons: step ranges of an uneven batch read back
    as the oracle's raster cut to them, after snn_log_clear the log restarts
    at the current step, and when instances fill their shares the readout
    counts the spikes kept (each instance's own up to its share) and reports
    SNN_E_OVERFLOW."""
    import ctypes
    prob = si.batched_sweep(n_nets=12, base_seed=3, n_steps=1500, n_lo=37, n_hi=6000)
    o = oracle_run("batch12", prob)
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=prob.n * 1500)
    try:
        net.step(600)
        for t0, t1 in [(0, 600), (0, 1), (137, 138), (250, 599), (599, 10_000), (600, 700)]:
            s, i = net.spikes(t0, t1)
            m = (o["steps"] >= t0) & (o["steps"] < min(t1, 600))
            assert np.array_equal(s, o["steps"][m]) and np.array_equal(i, o["ids"][m]), (t0, t1)
        net.log_clear()
        net.step(400)
        s, i = net.spikes()
        m = (o["steps"] >= 600) & (o["steps"] < 1000)
        assert len(i) > 0 and np.array_equal(s, o["steps"][m]) and np.array_equal(i, o["ids"][m])
    finally:
        net.close()
    cap = prob.n * 15  # 15 spikes per neuron: the busier instances (up to 27) overflow within 1,500 steps
    sizes = np.diff(prob.inst_off.astype(np.int64))
    share = cap * sizes // int(sizes.sum())
    per_inst = np.bincount(np.searchsorted(prob.inst_off[1:], o["ids"], side="right"), minlength=len(sizes))
    kept = np.minimum(per_inst, share)
    assert (per_inst > share).any() and (per_inst < share).any()
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=cap)
    try:
        net.step(1500)
        with pytest.raises(gpu.SnnError) as ei:
            net.sync()
        assert ei.value.status == -4
        n = ctypes.c_uint64(0)
        st = net.lib.snn_read_spikes(net.ctx, 0, 2**32 - 1, None, None, 0, ctypes.byref(n))
        assert st == -4 and n.value == int(kept.sum())
    finally:
        net.close()


def test_reset_repeats_the_run(gpu):
    prob = si.brunel_stdp_100k(seed=5, n_steps=600, n=2000, k=200)
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=1 << 20)
    net.step(600)
    a = net.spikes()
    wa = net.read("w")
    net.reset()
    net.step(600)
    b = net.spikes()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert np.array_equal(wa, net.read("w"))
    net.close()


@pytest.mark.parametrize("packed", [True, False])
def test_weight_write_reaches_the_receive(gpu, packed):
    """Weights written through the ABI are the ones the tiled receive
    delivers: the sweep's rows each carry one weight, so the receive reads
    16-bit target offsets and the row weights (2 bytes per event); weights
    that differ inside a row switch it to the packed edges (offset and code,
    4 bytes), rebuilt from them."""
    import dataclasses
    prob = si.batched_sweep(n_nets=4, base_seed=3, n_steps=300, n_lo=500, n_hi=3000)
    w = prob.w.copy()
    w[::3] = 0
    w[1::7] = -w[1::7]
    changed = dataclasses.replace(prob, w=w)
    o = oracle.run(changed)
    net = gpu.Network(prob, receive=RECV["tiled"], log_capacity=prob.n * 300, packed=packed)
    assert net.info()["edge_bytes"] == (2 if packed else 6)
    net.write("w", w)
    assert net.info()["edge_bytes"] == (4 if packed else 6)
    net.step(300)
    g = {f: net.read(f) for f in _fields(prob)}
    g["steps"], g["ids"] = net.spikes()
    g["counters"] = net.counters()
    net.close()
    assert len(o["ids"]) > 1000
    assert_parity(g, o, changed)


def test_stats_match_raster(gpu):
    """The binary64 device reductions equal rate and ISI CV computed from
    the raster."""
    prob = si.brunel_12k5(seed=2, n_steps=2000)
    net = gpu.Network(prob, stats=True, log_capacity=1 << 22)
    net.step(200)
    net.stats_clear()
    net.step(1800)
    rate, cv = net.stats(0)
    steps, ids = net.spikes(200, 2000)
    net.close()
    assert abs(rate - len(ids) / prob.n / 0.18) < 1e-9 * rate
    order = np.lexsort((steps, ids))
    s, i = steps[order].astype(np.float64), ids[order]
    starts = np.flatnonzero(np.r_[True, i[1:] != i[:-1]])
    ends = np.r_[starts[1:], len(i)]
    cvs = [np.diff(s[a:b]).std() / np.diff(s[a:b]).mean() for a, b in zip(starts, ends) if b - a >= 3]
    assert abs(cv - np.mean(cvs)) < 1e-9


@pytest.mark.parametrize("receive", ["tiled", "bulk"])
@pytest.mark.parametrize("tune_steps", [1, 37])
def test_retuned_tiles_keep_parity(gpu, tune_steps, receive):
    """Re-cutting the tiles by measured work mid-run changes nothing."""
    prob = si.batched_sweep(n_nets=9, base_seed=8, n_steps=400, n_lo=200, n_hi=20000)
    o = oracle_run("batch9", prob)
    net = gpu.Network(prob, receive=RECV[receive], log_capacity=prob.n * 400, tune_steps=tune_steps)
    before = net.info()["n_tiles"]
    for k in (10, 50, 340):
        net.step(k)
    after = net.info()["n_tiles"]
    g = {f: net.read(f) for f in _fields(prob)}
    g["steps"], g["ids"] = net.spikes()
    g["counters"] = net.counters()
    net.close()
    assert before > 0 and after > 0
    assert_parity(g, o, prob)


@pytest.mark.parametrize("packed", [True, False])
@pytest.mark.parametrize("n_inst,delay", [(1, 1), (2, 2), (3, 1), (33, 2), (1100, 2), (1, 3), (33, 3), (1100, 5)])
def test_per_step_plan_tile_counts(gpu, n_inst, delay, packed):
    """The tiled receive's per-step plan over 1 to 1,100 tiles (its rank sort
    up to 1,024 tiles, its sorting network above), with the plan beside the
    update (delay 2), before the receive (delay 1), and made one step ahead
    inside the fused step kernel (delays 3 and 5)."""
    insts = [si.brunel_instance(200 + 37 * (b % 7), k=20 + (b % 5), nu_ratio=3.0, graph_seed=b + 1)
             for b in range(n_inst)]
    prob = si.problem(si.BRUNEL, insts, delay=delay, n_steps=80, seed=7)
    o = oracle_run(("plan", n_inst, delay), prob)
    g = run_gpu(gpu, prob, w16=True, receive="tiled", packed=packed)
    assert len(o["ids"]) > 10 * n_inst
    assert_parity(g, o, prob)


@pytest.mark.parametrize("receive", ["tiled", "bulk"])
@pytest.mark.parametrize("model", [si.BRUNEL, si.VOGELS])
def test_instances_larger_than_one_tile(gpu, model, receive):
    """Instances whose accumulators exceed one CTA's shared memory are cut
    into target tiles; row segments come from the split table."""
    if model == si.BRUNEL:
        prob = si.problem(si.BRUNEL, [si.brunel_instance(70000, k=60, nu_ratio=3.0),
                                      si.brunel_instance(3000, k=300)], delay=3, n_steps=300, seed=4)
    else:
        prob = si.problem(si.VOGELS, [si.vogels_instance(31000, k=80, c=1.0)], delay=1, n_steps=300, seed=4)
    o = oracle.run(prob)
    net = gpu.Network(prob, receive=RECV[receive], log_capacity=prob.n * 300, tune_steps=100)
    net.step(300)
    info = net.info()
    g = {f: net.read(f) for f in _fields(prob)}
    g["steps"], g["ids"] = net.spikes()
    g["counters"] = net.counters()
    net.close()
    assert info["n_tiles"] >= 2
    assert len(o["ids"]) > 1000
    assert_parity(g, o, prob)


def form_of(info) -> str:
    """The receive form a context runs, in snn_info.tune_ms's names."""
    return "fused" if info["fused"] else info["receive"]


def assert_tuned_fastest(info):
    """SNN_RECV_AUTO kept the form its timing run measured fastest."""
    assert info["tuned"]
    ms = {k: v for k, v in info["tune_ms"].items() if v > 0}
    assert len(ms) >= 1 and form_of(info) in ms
    assert form_of(info) == min(ms, key=ms.get), (form_of(info), ms)


@pytest.mark.parametrize("name,n_steps", [("vogels_4k", 1000), ("brunel_12k5", 2000), ("brunel_stdp_100k", 300)])
def test_tuned_receive_is_the_measured_fastest(gpu, name, n_steps):
    """SNN_RECV_AUTO times every form that applies on the graph itself and
    keeps the fastest (snn_info.tune_ms); the run that follows starts from
    N_0 and equals the oracle's (the tuning steps leave no trace)."""
    prob = getattr(si, name)(seed=1, n_steps=n_steps)
    net = gpu.Network(prob, receive=0, log_capacity=prob.n * n_steps + 4096)
    try:
        info = net.info()
        assert_tuned_fastest(info)
        # the generator sorts rows: both the global and the tiled form were timed
        assert info["tune_ms"]["tiled"] > 0 and info["tune_ms"]["global"] > 0
        net.step(n_steps)
        g = {f: net.read(f) for f in _fields(prob)}
        g["steps"], g["ids"] = net.spikes()
        g["counters"] = net.counters()
    finally:
        net.close()
    assert_parity(g, oracle_run(("tuned", name, n_steps), prob), prob)


def test_bulk_wait_bound_reports_timeout(gpu):
    """The bulk receive's producer and consumer waits are bounded: with a
    bound of one poll a chunk's copy is not yet in shared memory when its
    consumer first looks, the wait gives up, and the kernel drains the copies
    it issued (under its own, large bound) before its CTAs exit.  The step
    reports SNN_E_TIMEOUT through snn_sync, the CUDA context stays usable
    (reset and stepping again raise no CUDA error), and a context with the
    default bound on the same device still matches the oracle."""
    prob = si.batched_sweep(n_nets=3, base_seed=4, n_steps=60, n_lo=2000, n_hi=6000)
    net = gpu.Network(prob, receive=RECV["bulk"], log_capacity=1 << 20, wait_polls=1)
    try:
        net.step(prob.n_steps)
        with pytest.raises(gpu.SnnError) as e:
            net.sync()
        assert e.value.status == -5  # SNN_E_TIMEOUT
        net.reset()  # clears the error; the device answers
        net.step(prob.delay + 10)  # past the delay: spikes are delivered again
        with pytest.raises(gpu.SnnError) as e:
            net.sync()
        assert e.value.status == -5
    finally:
        net.close()
    ref = oracle.run(prob)
    out = run_gpu(gpu, prob, receive="bulk")
    assert np.array_equal(out["steps"], ref["steps"]) and np.array_equal(out["ids"], ref["ids"])
    assert len(ref["ids"]) > 0


def test_row_weight_layout(gpu):
    """Rows that carry one weight each (the source population's: Vogels and
    Brunel, Section III-A-2 and Table 2) let the global receive read the
    4-byte targets alone; SNN_F_UNPACKED keeps the per-edge codes (6 bytes).
    Writing weights that differ inside a row switches the receive back to the
    per-edge codes, and the run still equals the oracle's on those weights."""
    prob = si.vogels_4k(seed=2, n_steps=400)
    o = oracle_run("v4k_s2", prob)
    for packed, eb in ((True, 4), (False, 6)):
        net = gpu.Network(prob, receive=RECV["global"], log_capacity=prob.n * 400, packed=packed)
        try:
            assert net.info()["edge_bytes"] == eb
            net.step(prob.n_steps)
            g = {f: net.read(f) for f in _fields(prob)}
            g["steps"], g["ids"] = net.spikes()
            g["counters"] = net.counters()
        finally:
            net.close()
        assert_parity(g, o, prob)
    # 200 excitatory rows get a second weight value in their first edge
    # (same shift: 2^2 x 32767, 2.0 mV against 1.62 mV)
    w2 = prob.w.copy()
    for j in range(200):
        a = int(prob.row_off[j])
        assert int(prob.row_off[j + 1]) - a >= 2 and w2[a] == 106168
        w2[a] = 131068
    prob2 = si.Problem(model=prob.model, instances=prob.instances, delay=prob.delay, seed=prob.seed,
                       n_steps=prob.n_steps, stdp=False, inst_off=prob.inst_off, row_off=prob.row_off,
                       tgt=prob.tgt, w=w2)
    o2 = oracle.run(prob2)
    net = gpu.Network(prob, receive=RECV["global"], log_capacity=prob.n * 400)
    try:
        assert net.info()["edge_bytes"] == 4
        net.write("w", w2)
        assert net.info()["edge_bytes"] == 6
        net.step(prob.n_steps)
        g = {f: net.read(f) for f in _fields(prob)}
        g["steps"], g["ids"] = net.spikes()
        g["counters"] = net.counters()
        assert np.array_equal(net.read("w"), w2)
    finally:
        net.close()
    assert_parity(g, o2, prob2)
    assert not np.array_equal(o2["ids"], o["ids"])  # the changed weight matters


def test_persistent_launch_chunks_and_barrier_timeout(gpu):
    """The persistent launch runs each snn_step call as one cooperative
    launch: a run cut into calls of 1, 7 and 250 steps equals the oracle.  Its
    grid-barrier waits are bounded: with a bound of one poll every CTA but the
    last to arrive gives up, the launch ends with SNN_E_TIMEOUT, and the
    context resets and the device answers."""
    prob = si.vogels_4k(seed=3, n_steps=600)
    o = oracle_run("v4k_s3", prob)
    net = gpu.Network(prob, receive=RECV["persistent"], log_capacity=prob.n * 600)
    try:
        info = net.info()
        assert info["persistent"] and info["persist_ctas"] >= 2
        for k in (1, 7, 250, 342):
            net.step(k)
        g = {f: net.read(f) for f in _fields(prob)}
        g["steps"], g["ids"] = net.spikes()
        g["counters"] = net.counters()
    finally:
        net.close()
    assert_parity(g, o, prob)
    net = gpu.Network(prob, receive=RECV["persistent"], log_capacity=prob.n * 600, wait_polls=1)
    try:
        net.step(50)
        with pytest.raises(gpu.SnnError) as e:
            net.sync()
        assert e.value.status == -5  # SNN_E_TIMEOUT
        net.reset()
        net.step(1)
        with pytest.raises(gpu.SnnError) as e:
            net.sync()
        assert e.value.status == -5
    finally:
        net.close()
