"""Pins of the CPU oracle against things other than itself.

Each test ties one part of the oracle to a library routine, a closed form,
an exact timing property of the pipeline (Section III-A-1, Fig. 1) or a
brute-force computation, so that a dropped term, a wrong sign, a swapped
index or an off-by-one step fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.stats

import oracle
import snn_inputs as si


def _graph(n, edges, w):
    """CSR input from an explicit edge list [(src, tgt)] with weights."""
    order = sorted(range(len(edges)), key=lambda k: edges[k])
    row_off = np.zeros(n + 1, np.uint64)
    for s, _ in edges:
        row_off[s + 1] += 1
    row_off = np.cumsum(row_off).astype(np.uint64)
    tgt = np.array([edges[k][1] for k in order], np.uint32)
    ww = np.array([w[k] for k in order], np.int32)
    return row_off, tgt, ww


def _problem(model, inst, n_steps, delay=1, edges=(), w=(), stdp=False, seed=7):
    row_off, tgt, ww = _graph(inst.n, list(edges), list(w))
    return si.Problem(model=model, instances=[inst], delay=delay, seed=seed, n_steps=n_steps, stdp=stdp,
                      inst_off=np.array([0, inst.n], np.uint32), row_off=row_off, tgt=tgt, w=ww)


def _state(n, E=0, **kw):
    st = {"V": np.zeros(n, np.float32), "ge": np.zeros(n, np.float32), "gi": np.zeros(n, np.float32),
          "r": np.zeros(n, np.int32), "x": np.zeros(n, np.float32), "y": np.zeros(n, np.float32),
          "acc0": np.zeros(n, np.int32), "acc1": np.zeros(n, np.int32), "w": np.zeros(E, np.int32)}
    for k, v in kw.items():
        if k == "w":
            st[k] = np.asarray(v, np.int32).copy()
        else:
            st[k][...] = v
    return st


# ---------------------------------------------------------------- Philox
@pytest.mark.parametrize("ctr,key", [((1, 0, 0, 0), (0, 0)), ((5, 7, 1, 0), (123, 456)),
                                     ((2**63 + 11, 2**64 - 1, 3, 2**40), (2**64 - 5, 99)),
                                     ((9, 10000, 1, 0), (1, 255))])
def test_philox_matches_numpy(ctr, key):
    """Philox4x64-10 against numpy's bit generator (which advances the
    counter once before its first block)."""
    g = np.random.Philox(counter=np.array([ctr[0] - 1, *ctr[1:]], dtype=np.uint64),
                         key=np.array(key, dtype=np.uint64))
    ref = g.random_raw(4)
    got = oracle.philox4x64_10(ctr, key)
    assert list(got) == list(ref)


def test_rand_word_is_the_documented_half():
    """Word (local & 7) of the block at counter (local >> 3, step, tag, 0),
    low half first, key (seed, instance); checked against numpy's Philox."""
    seed, inst, step, tag = 42, 3, 17, 1
    for local in [0, 1, 2, 7, 8, 13, 1000003]:
        c0 = local >> 3
        g = np.random.Philox(counter=np.array([c0 - 1 if c0 else 2**64 - 1, step - (0 if c0 else 1), tag, 0],
                                              dtype=np.uint64), key=np.array([seed, inst], dtype=np.uint64))
        blk = g.random_raw(4)
        wsel = local & 7
        ref = (int(blk[wsel >> 1]) >> (32 * (wsel & 1))) & 0xFFFFFFFF
        assert oracle.rand_word(seed, inst, local, step, tag) == ref


# ---------------------------------------------------------------- Poisson
@pytest.mark.parametrize("lam", [0.0, 0.5, 0.9, 2.0, 4.0, 12.5])
def test_poisson_table_matches_scipy_cdf(lam):
    T = oracle.poisson_table(lam)
    k = np.arange(len(T))
    cdf = scipy.stats.poisson.cdf(k, lam)
    assert np.all(np.abs(T.astype(np.float64) / 2**32 - cdf) <= 2.0**-32 + 1e-13)
    # the table stops where the remaining tail is below 2^-32
    assert scipy.stats.poisson.sf(len(T), lam) < 1e-9 if lam > 0 else len(T) == 0


@pytest.mark.parametrize("lam", [0.9, 2.0, 4.0])
def test_poisson_sampler_distribution(lam):
    T = oracle.poisson_table(lam)
    u = np.random.Generator(np.random.PCG64(5)).integers(0, 2**32, size=400_000, dtype=np.uint64)
    # vectorised form of #{k : T_k <= u}, checked against the C sampler on a subset
    x = np.searchsorted(T.astype(np.uint64), u, side="right")
    for uu, xx in zip(u[:200], x[:200]):
        assert oracle.poisson_sample(T, int(uu)) == xx
    assert abs(x.mean() - lam) < 5 * math.sqrt(lam / len(x))
    assert abs(x.var() - lam) < 0.02 * lam + 5 * math.sqrt(2 * lam * lam / len(x))
    kmax = int(lam + 6 * math.sqrt(lam) + 2)
    obs = np.bincount(np.minimum(x, kmax), minlength=kmax + 1)
    p = scipy.stats.poisson.pmf(np.arange(kmax + 1), lam)
    p[-1] = scipy.stats.poisson.sf(kmax - 1, lam)
    keep = p * len(x) > 20
    chi2 = (((obs - p * len(x)) ** 2) / (p * len(x)))[keep].sum()
    assert chi2 < scipy.stats.chi2.ppf(0.9999, keep.sum() - 1)


# ---------------------------------------------------------------- LIF closed forms
def test_vogels_time_to_threshold_and_period():
    """No synapses, constant drive E_L = -49 mV: V_n = E_L + (V0-E_L) Pm^n,
    so the first spike comes after ceil(ln((V0-E_L)/(V_th-E_L)) / (dt/tau))
    updates, then every R + n*(V_reset) updates (n*(-60) = 480, R = 50)."""
    inst = si.vogels_instance(64)
    rng = np.random.Generator(np.random.PCG64(3))
    V0 = np.concatenate([[-60.0], rng.uniform(-60.0, -50.2, 63)]).astype(np.float32)
    p = _problem(si.VOGELS, inst, n_steps=2000, edges=())
    out = oracle.run(p, state=_state(64, V=V0))
    rate = inst.dt / inst.tau_m
    n_reset = math.ceil(math.log((inst.v_reset - inst.e_l) / (inst.v_th - inst.e_l)) / rate)
    assert n_reset == 480
    checked = 0
    for i in range(64):
        real = math.log((float(V0[i]) - inst.e_l) / (inst.v_th - inst.e_l)) / rate
        if abs(real - round(real)) < 0.05:
            continue  # too close to a step boundary for binary32
        first = math.ceil(real) - 1  # update index t produces V_{t+1}
        expect = [first]
        while expect[-1] + inst.refractory_steps + n_reset < 2000:
            expect.append(expect[-1] + inst.refractory_steps + n_reset)
        got = out["steps"][out["ids"] == i]
        assert list(got) == expect, (i, V0[i])
        checked += 1
    assert checked > 40


def test_brunel_leak_closed_form():
    """No input, no drive: V_t = V0 Pm^t with Pm = exp(-dt/tau)."""
    inst = si.brunel_instance(16, k=0)
    inst.lam = 0.0
    inst.v_th = 1e9
    V0 = np.linspace(1.0, 19.0, 16).astype(np.float32)
    for T in (1, 10, 700):
        out = oracle.run(_problem(si.BRUNEL, inst, n_steps=T), state=_state(16, V=V0))
        ref = V0.astype(np.float64) * math.exp(-inst.dt / inst.tau_m) ** T
        assert np.allclose(out["V"], ref, rtol=T * 2.0**-23 + 1e-7, atol=0)


def test_brunel_poisson_drive_mean_and_variance():
    """Subthreshold Brunel neurons under Poisson drive only: the membrane is
    a filtered compound Poisson process, E[V_t] = lam J (1-Pm^t)/(1-Pm) and
    Var[V_t] = lam J^2 (1-Pm^2t)/(1-Pm^2)."""
    n, T = 20000, 300
    inst = si.brunel_instance(n, k=0, nu_ratio=2.0)
    inst.v_th = 1e9
    out = oracle.run(_problem(si.BRUNEL, inst, n_steps=T, seed=11), state=_state(n))
    Pm = math.exp(-inst.dt / inst.tau_m)
    J = inst.jext_q / 65536.0
    mean = inst.lam * J * (1 - Pm**T) / (1 - Pm)
    var = inst.lam * J * J * (1 - Pm ** (2 * T)) / (1 - Pm * Pm)
    V = out["V"].astype(np.float64)
    assert abs(V.mean() - mean) < 5 * math.sqrt(var / n)
    assert abs(V.var() / var - 1) < 0.05


# ---------------------------------------------------------------- delay FIFO
@pytest.mark.parametrize("d", [1, 2, 15, 16])
@pytest.mark.parametrize("src", [0, 3])  # 0 excitatory, 3 inhibitory (n_exc = 3)
def test_fifo_exact_arrival_vogels(d, src):
    """A spike of step tau reaches its targets' update at step tau + d
    exactly (Receive reads S_{t-d+1}; the update after it sees the input),
    and lands on ge for an excitatory source, gi for an inhibitory one."""
    inst = si.vogels_instance(5)
    inst.n_exc = 3
    tau = 4
    w = 106168 if src == 0 else -589824
    edges = [(src, 1), (src, 2)]
    for T in range(tau + d - 1, tau + d + 2):
        p = _problem(si.VOGELS, inst, n_steps=T + 1, delay=d, edges=edges, w=[w, w])
        V0 = np.full(5, -60.0, np.float32)
        out = oracle.run(p, overrides=[(tau, src, 1000.0)], state=_state(5, V=V0, w=[w, w]))
        assert list(out["ids"][out["steps"] == tau]) == [src]
        ch, other = ("ge", "gi") if src == 0 else ("gi", "ge")
        steps_run = T + 1
        arrived = steps_run - 1 >= tau + d  # last update index is T
        exp = 0.0
        # the update at step tau+d adds the input then decays it once
        if arrived:
            k = (T - (tau + d))
            exp = (w / 65536.0) * math.exp(-inst.dt / (inst.tau_e if src == 0 else inst.tau_i)) ** (k + 1)
        assert np.allclose(out[ch][[1, 2]], exp, rtol=1e-5, atol=0)
        assert np.all(out[other][[1, 2]] == 0)
        # pending input: delivered by the receive of update index tau+d-1
        pend = out["acc0" if src == 0 else "acc1"][[1, 2]]
        assert list(pend) == ([w, w] if T == tau + d - 1 else [0, 0])


@pytest.mark.parametrize("d", [1, 2, 15])
def test_fifo_exact_arrival_brunel(d):
    inst = si.brunel_instance(4, k=0)
    inst.lam = 0.0
    inst.n_exc = 2
    tau = 3
    w = 6554
    for T in range(tau + d - 1, tau + d + 1):
        p = _problem(si.BRUNEL, inst, n_steps=T + 1, delay=d, edges=[(0, 1), (0, 3)], w=[w, w])
        out = oracle.run(p, overrides=[(tau, 0, 100.0)], state=_state(4, w=[w, w]))
        if T == tau + d - 1:
            assert list(out["acc0"]) == [0, w, 0, w] and out["V"][1] == 0.0
        else:
            assert out["V"][1] == np.float32(w / 65536.0) and out["V"][3] == np.float32(w / 65536.0)


# ---------------------------------------------------------------- relay (ping-pong) network
def _relay_problem(n_a, n_b, p, d, n_steps, seed):
    """Listing 1's ping_pong model in LIF form: no leak memory (Pm = 0),
    threshold below one synaptic weight, no refractory period, no drive, so
    a neuron spikes exactly when it received a spike in the previous
    delivery: S_{t+d} = out-neighbours(S_t)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = n_a + n_b
    edges = []
    for j in range(n_a):
        for i in range(n_a, n):
            if rng.random() < p:
                edges.append((j, i))
    for j in range(n_a, n):
        for i in range(n_a):
            if rng.random() < p:
                edges.append((j, i))
    inst = si.brunel_instance(n, k=0)
    inst.n_exc = n
    inst.tau_m = 1e-6
    inst.v_th = 0.05
    inst.v_reset = 0.0
    inst.refractory_steps = 0
    inst.lam = 0.0
    w = [6554] * len(edges)
    prob = _problem(si.BRUNEL, inst, n_steps=n_steps, delay=d, edges=edges, w=w)
    return prob, edges


@pytest.mark.parametrize("d", [1, 3])
def test_relay_network_matches_bfs(d):
    n_a = n_b = 100
    prob, edges = _relay_problem(n_a, n_b, 0.05, d, 40, seed=1)
    succ = {j: set() for j in range(n_a + n_b)}
    for j, i in edges:
        succ[j].add(i)
    acc0 = np.zeros(n_a + n_b, np.int32)
    acc0[:n_a] = 6554  # population A received a spike before step 0
    out = oracle.run(prob, state=_state(n_a + n_b, acc0=acc0, w=[6554] * len(edges)))
    frontier = set(range(n_a))
    expect = {0: frontier}
    t = 0
    while t + d < 40:
        frontier = set().union(*[succ[j] for j in frontier]) if frontier else set()
        t += d
        expect[t] = frontier
    assert any(len(v) for k, v in expect.items() if k > 10)
    for t in range(40):
        got = set(out["ids"][out["steps"] == t].tolist())
        assert got == expect.get(t, set()), t


# ---------------------------------------------------------------- dense brute force
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_receive_matches_dense_matmul(seed):
    """Receive Spikes over a CSR equals W^T s for the dense weight matrix,
    split by the source's population (two input channels in Vogels)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 47
    inst = si.vogels_instance(n)
    inst.n_exc = 30
    mask = rng.random((n, n)) < 0.3
    np.fill_diagonal(mask, False)
    edges = [(j, i) for j in range(n) for i in range(n) if mask[j, i]]
    w = rng.integers(-2**20, 2**20, size=len(edges)).tolist()
    p = _problem(si.VOGELS, inst, n_steps=1, edges=edges, w=w)
    W = np.zeros((n, n), np.int64)
    for (j, i), ww in zip(edges, w):
        W[j, i] = ww
    for _ in range(5):
        s = np.flatnonzero(rng.random(n) < 0.4)
        a0, a1, ev = oracle.receive(p, s)
        x = np.zeros(n, np.int64)
        x[s] = 1
        xe, xi = x.copy(), x.copy()
        xe[inst.n_exc:] = 0
        xi[:inst.n_exc] = 0
        assert np.array_equal(a0, W.T @ xe)
        assert np.array_equal(a1, W.T @ xi)
        assert ev == int(mask[s].sum())


# ---------------------------------------------------------------- STDP closed form
def _stdp_pair(pre_steps, post_steps, d, w0, n_steps=None):
    inst = si.brunel_instance(2, k=0, stdp=True)
    inst.n_exc = 2
    inst.lam = 0.0
    inst.v_th = 1000.0
    inst.refractory_steps = 0
    last = max(list(pre_steps) + list(post_steps)) + d + 2
    p = _problem(si.BRUNEL, inst, n_steps=n_steps or last, delay=d, edges=[(0, 1)], w=[w0], stdp=True)
    ov = [(t, 0, 1e5) for t in pre_steps] + [(t, 1, 1e5) for t in post_steps]
    out = oracle.run(p, overrides=ov, state=_state(2, E=1, w=[w0]))
    assert sorted(out["steps"][out["ids"] == 0].tolist()) == sorted(pre_steps)
    assert sorted(out["steps"][out["ids"] == 1].tolist()) == sorted(post_steps)
    return out["w"][0], inst


@pytest.mark.parametrize("delta", [0, 1, 5, 40, -1, -7, -40])
@pytest.mark.parametrize("d", [1, 15])
def test_stdp_single_pair_closed_form(delta, d):
    """One pre spike arriving at t_arr = t_pre + d and one post spike at
    t_post: dw = A+ w_max exp(-delta dt/tau+) for delta = t_post - t_arr >= 0
    (coincidence counts as causal), A- w_max exp(delta dt/tau-) otherwise,
    rounded to the lattice."""
    w0 = 6554
    t_pre = 50
    t_post = t_pre + d + delta
    w, inst = _stdp_pair([t_pre], [t_post], d, w0)
    if delta >= 0:
        ref = inst.a_plus * inst.w_max_q * math.exp(-delta * inst.dt / inst.tau_plus)
    else:
        ref = inst.a_minus * inst.w_max_q * math.exp(delta * inst.dt / inst.tau_minus)
    assert abs((int(w) - w0) - ref) <= 1.0
    assert (int(w) - w0 > 0) == (delta >= 0)


def test_stdp_all_to_all_additive_and_clipping():
    d = 2
    # two pre arrivals before one post spike: the traces add
    w, inst = _stdp_pair([10, 14], [30], d, 6554)
    Ap = inst.a_plus * inst.w_max_q
    ref = Ap * (math.exp(-(30 - 12) * inst.dt / 20.0) + math.exp(-(30 - 16) * inst.dt / 20.0))
    assert abs((int(w) - 6554) - ref) <= 1.0
    # potentiation is clipped at w_max, depression at 0
    w, inst = _stdp_pair([10], [12], d, inst.w_max_q - 3)
    assert w == inst.w_max_q
    w, inst = _stdp_pair([20], [5], d, 40)
    assert w == 0


# ---------------------------------------------------------------- whole-run invariants
def test_vogels_run_invariants():
    p = si.vogels_4k(seed=2, n_steps=600)
    out = oracle.run(p)
    steps, ids = out["steps"], out["ids"]
    assert len(ids) > 100
    # sorted by (step, id)
    key = steps.astype(np.int64) * p.n + ids
    assert np.all(np.diff(key) > 0)
    # refractoriness: consecutive spikes of a neuron are > R steps apart
    order = np.lexsort((steps, ids))
    s_ids, s_steps = ids[order], steps[order]
    same = s_ids[1:] == s_ids[:-1]
    assert np.all(np.diff(s_steps.astype(np.int64))[same] > 50)
    # delivered events = sum of the out-degrees of the delivered spikes
    deg = np.diff(p.row_off.astype(np.int64))
    assert out["events"] == int(deg[ids].sum())  # d = 1: every spike before the last step is delivered


# ---------------------------------------------------------------- Init stage (V0 draw)
def _numpy_words(seed, inst, local, step, tag):
    """The 32-bit word of neuron `local` from numpy's own Philox4x64-10: the
    block at counter (local >> 3, step, tag, 0), key (seed, inst); word
    local & 7, low half of each 64-bit output first."""
    # numpy advances its 256-bit counter once before the first block
    c = ((local >> 3) | step << 64 | tag << 128) - 1
    c %= 1 << 256
    g = np.random.Philox(counter=np.array([(c >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64),
                         key=np.array([seed, inst], dtype=np.uint64))
    raw = g.random_raw(4)
    k = local & 7
    return int(raw[k // 2]) >> (32 * (k % 2)) & 0xffffffff


@pytest.mark.parametrize("model", [si.VOGELS, si.BRUNEL])
def test_initial_potential_draw(model):
    """The Init stage (Fig. 1: N -> N_0) draws V0 = v0_lo + v0_span u with
    u = (w >> 8) 2^-24 from the tag-0, step-0 Philox word of each neuron,
    keyed by (seed, instance).  The words come from numpy's Philox, not the
    oracle's; the uniform law of V0 over [v0_lo, v0_lo + v0_span) is checked
    against the configured range (a wrong span, offset, word, step, tag or
    instance key fails one of the two checks).  Zero steps: N_0 itself."""
    n = 600
    if model == si.VOGELS:
        insts = [si.vogels_instance(n, k=0) for _ in range(3)]
    else:
        insts = [si.brunel_instance(n, k=0) for _ in range(3)]
    seed = 12345
    lo, span = insts[0].v0_lo, insts[0].v0_span
    assert (lo, span) == ((-60.0, 10.0) if model == si.VOGELS else (0.0, 20.0))
    p = si.Problem(model=model, instances=insts, delay=1, seed=seed, n_steps=0, stdp=False,
                   inst_off=np.arange(4, dtype=np.uint32) * n, row_off=np.zeros(3 * n + 1, np.uint64),
                   tgt=np.zeros(0, np.uint32), w=np.zeros(0, np.int32))
    for key0 in (0, 7):  # the instance key may start at another index (one network of a batch re-run alone)
        out = oracle.run(p, inst_key0=key0)
        V = out["V"]
        for b in range(3):
            for local in list(range(0, 40)) + list(range(n - 24, n)):
                w = _numpy_words(seed, key0 + b, local, 0, 0)
                u = np.float32(w >> 8) * np.float32(2.0 ** -24)
                expect = np.float32(lo) + np.float32(span) * u
                assert V[b * n + local] == expect, (b, local)
        assert np.all(V >= lo) and np.all(V < lo + span)
        # uniform on the range: mean and variance within 5 standard errors
        x = (V.astype(np.float64) - lo) / span
        assert abs(x.mean() - 0.5) < 5 * math.sqrt(1 / 12 / V.size)
        assert abs(x.var() - 1 / 12) < 5 * math.sqrt(1 / 180 / V.size)
        assert scipy.stats.kstest(x, "uniform").pvalue > 1e-4
        # instances draw independently: different keys, different potentials
        assert not np.array_equal(V[:n], V[n:2 * n])
    assert np.all(out["r"] == 0) and np.all(out["acc0"] == 0) and np.all(out["ge"] == 0)


# ---------------------------------------------------------------- Brunel refractory clamp
def test_brunel_refractory_period_and_discarded_input():
    """Brunel neuron (Section IV), R = 20 steps: held far above threshold
    before every update it fires every R + 1 steps -- the clamp covers the R
    updates after a spike, at which V = V_reset and the input is discarded.
    A synaptic input delivered inside the clamp is dropped: after the clamp
    ends the neuron starts again from V_reset and does not fire on it, while
    the same input arriving after the clamp makes it fire."""
    inst = si.brunel_instance(3, k=0)
    inst.lam = 0.0
    inst.n_exc = 3
    R = inst.refractory_steps
    assert R == 20
    # (a) period under a constant forced supra-threshold drive
    T = 200
    p = _problem(si.BRUNEL, inst, n_steps=T, delay=1)
    out = oracle.run(p, overrides=[(t, 0, 1000.0) for t in range(T)], state=_state(3))
    got = list(out["steps"][out["ids"] == 0])
    assert got == list(range(0, T, R + 1))
    # V at the end of each clamped step is V_reset exactly
    for Tend in (1, 5, R, R + 1):
        o = oracle.run(_problem(si.BRUNEL, inst, n_steps=Tend, delay=1), overrides=[(0, 0, 1000.0)],
                       state=_state(3))
        assert o["V"][0] == np.float32(inst.v_reset)
        assert o["r"][0] == (R - (Tend - 1) if Tend <= R + 1 else 0)
    # (b) input inside the clamp is discarded.  Neuron 1 -> 0 with a weight
    # that alone crosses threshold from V_reset; neuron 1 is forced to fire
    # at step s, its spike reaches neuron 0's update at step s + 1 (d = 1).
    w = quantize = int(round(30.0 * 65536))  # 30 mV: V_reset * Pm + 30 > theta
    assert quantize == w
    for s, fires in ((3, False), (R - 1, False), (R, True), (R + 5, True)):
        p = _problem(si.BRUNEL, inst, n_steps=R + 10, delay=1, edges=[(1, 0)], w=[w])
        o = oracle.run(p, overrides=[(0, 0, 1000.0), (s, 1, 1000.0)], state=_state(3, w=[w]))
        s0 = list(o["steps"][o["ids"] == 0])
        # neuron 0 fires at 0; the arrival at update s + 1 is inside the
        # clamp (updates 1..R) exactly when s + 1 <= R
        assert s0 == ([0, s + 1] if fires else [0]), (s, s0)
        if not fires:
            # V after the clamp: V_reset decayed by the free updates since
            Pm = np.float32(math.exp(-inst.dt / inst.tau_m))
            v = np.float32(inst.v_reset)
            for _ in range(R + 10 - (R + 1)):
                v = np.float32(v * Pm) + np.float32(0.0)
            assert o["V"][0] == v
