"""Seeded synthetic inputs for the work-queue SNN timestep.

This module is shared by the oracle-side tests and the CUDA path and holds
none of the simulation's arithmetic: it only describes workloads (model
constants per network instance, connectivity, weights already on the
2^-16 mV lattice) and draws their random graphs.

The workloads stand in for the paper's benchmark models (Section IV): the
Vogels-Abbott CUBA network, the Brunel network with Poisson drive, Brunel
with STDP, each at several sizes, plus a batched sweep of many Brunel
networks.  There is no dataset; every graph comes from a seed.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_SO = os.path.join(_HERE, "libsnn_gen.so")
_lock = threading.Lock()
_lib = None

LATTICE = 65536  # lattice units per mV (weights are multiples of 2^-16 mV)
VOGELS, BRUNEL = 0, 1


def build(force: bool = False) -> str:
    """Compile the graph generator (plain C, pthreads)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread", "-o", _SO + ".tmp",
                               _SRC, "-lm"])
        os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            u32, u64, dbl, i32 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int32
            vp = ctypes.c_void_p
            lib.gen_bernoulli_count.restype = u64
            lib.gen_bernoulli_count.argtypes = [u64, u32, u32, dbl]
            lib.gen_bernoulli_fill.restype = None
            lib.gen_bernoulli_fill.argtypes = [u64, u32, u32, dbl, u32, u64, vp, vp]
            lib.gen_fixed_indegree.restype = ctypes.c_int
            lib.gen_fixed_indegree.argtypes = [u64, u32, u32, u32, u32, u32, u32, u64, vp, vp, ctypes.c_int]
            lib.gen_fill_weights.restype = None
            lib.gen_fill_weights.argtypes = [vp, u32, u32, i32, i32, vp]
            lib.gen_row_weights.restype = ctypes.c_int
            lib.gen_row_weights.argtypes = [vp, u32, vp, vp, ctypes.c_int]
            _lib = lib
    return _lib


def quantize_mV(w_mV: float) -> int:
    """Nearest value to w_mV (ties to even) that a 16-bit code times a power
    of two can hold on the 2^-16 mV lattice: q * 2^s with |q| <= 32767 and
    the smallest such s."""
    x = w_mV * LATTICE
    s = 0
    while True:
        q = round(x / (1 << s))  # Python rounds half to even
        if -32768 <= q <= 32767:
            return int(q) << s
        s += 1


@dataclasses.dataclass
class Instance:
    """One network: its size, population split and model constants."""
    n: int
    n_exc: int
    dt: float = 0.1
    tau_m: float = 20.0
    v_th: float = 20.0
    v_reset: float = 10.0
    refractory_steps: int = 20
    e_l: float = 0.0
    tau_e: float = 0.0
    tau_i: float = 0.0
    lam: float = 0.0
    jext_q: int = 0
    v0_lo: float = 0.0
    v0_span: float = 20.0
    tau_plus: float = 0.0
    tau_minus: float = 0.0
    a_plus: float = 0.0
    a_minus: float = 0.0
    w_max_q: int = 0
    # connectivity recipe
    p_conn: float = 0.0   # Bernoulli probability (0: fixed in-degree)
    k_exc: int = 0
    k_inh: int = 0
    w_exc_mV: float = 0.0
    w_inh_mV: float = 0.0
    graph_seed: int = 1

    @property
    def w_exc_q(self) -> int:
        return quantize_mV(self.w_exc_mV)

    @property
    def w_inh_q(self) -> int:
        return quantize_mV(self.w_inh_mV)


@dataclasses.dataclass
class Problem:
    """A whole simulation input: model, instances, graph, seed and length."""
    model: int
    instances: list
    delay: int
    seed: int
    n_steps: int
    stdp: bool = False
    inst_off: np.ndarray = None   # uint32 [B+1]
    row_off: np.ndarray = None    # uint64 [N+1]
    tgt: np.ndarray = None        # uint32 [E] global ids
    w: np.ndarray = None          # int32 [E] lattice units
    # one weight per row, with the weight array it was read from (row_weights)
    _w_row: np.ndarray = dataclasses.field(default=None, repr=False, compare=False)
    _w_row_of: object = dataclasses.field(default=None, repr=False, compare=False)

    @property
    def n(self) -> int:
        return int(self.inst_off[-1])

    @property
    def n_edges(self) -> int:
        return int(self.row_off[-1])

    def row_weights(self):
        """int32 [N]: the weight every synapse of row j carries, when each
        row carries one (the recipes here: one weight per source
        population), else None.  Read once per weight array: assign a new
        `w` rather than changing it in place."""
        if self.w is None or self.row_off is None:
            return None
        if self._w_row_of is self.w:
            return self._w_row
        n = len(self.row_off) - 1
        out = np.zeros(max(n, 1), dtype=np.int32)[:n]
        w = np.ascontiguousarray(self.w, dtype=np.int32)
        ro = np.ascontiguousarray(self.row_off, dtype=np.uint64)
        ok = _load().gen_row_weights(ro.ctypes.data, n, w.ctypes.data if w.size else None, out.ctypes.data,
                                     max(1, len(os.sched_getaffinity(0))))
        self._w_row, self._w_row_of = (out if ok else None), self.w
        return self._w_row

    def w_mV(self) -> np.ndarray:
        """Unquantised weights (mV, float64) for the binary64 comparison."""
        out = np.empty(self.n_edges, dtype=np.float64)
        for b, inst in enumerate(self.instances):
            lo, hi = int(self.inst_off[b]), int(self.inst_off[b + 1])
            ro = self.row_off
            e_mid = int(ro[lo + inst.n_exc])
            out[int(ro[lo]):e_mid] = inst.w_exc_mV
            out[e_mid:int(ro[hi])] = inst.w_inh_mV
        return out


def build_graph(prob: Problem, threads: int | None = None, inst_index0: int = 0) -> Problem:
    """Draw the connectivity of every instance and fill weights.  Instance b
    is drawn as instance inst_index0 + b of a batch (the index is part of
    its stream key), so network b of a batch can be rebuilt alone."""
    lib = _load()
    if threads is None:
        threads = max(1, len(os.sched_getaffinity(0)))
    sizes = [inst.n for inst in prob.instances]
    inst_off = np.zeros(len(sizes) + 1, dtype=np.uint32)
    inst_off[1:] = np.cumsum(sizes, dtype=np.uint64).astype(np.uint32)
    counts = []
    for b, inst in enumerate(prob.instances):
        if inst.p_conn > 0:
            counts.append(int(lib.gen_bernoulli_count(inst.graph_seed, inst_index0 + b, inst.n, inst.p_conn)))
        else:
            counts.append(inst.n * (inst.k_exc + inst.k_inh))
    E = int(sum(counts))
    N = int(inst_off[-1])
    row_off = np.zeros(N + 1, dtype=np.uint64)
    tgt = np.empty(max(E, 1), dtype=np.uint32)[:E]
    w = np.empty(max(E, 1), dtype=np.int32)[:E]
    ebase = 0
    for b, inst in enumerate(prob.instances):
        lo = int(inst_off[b])
        ro_ptr = row_off.ctypes.data + 8 * lo
        tg_ptr = tgt.ctypes.data + 4 * ebase
        if inst.p_conn > 0:
            lib.gen_bernoulli_fill(inst.graph_seed, inst_index0 + b, inst.n, inst.p_conn, lo, ebase, ro_ptr, tg_ptr)
        else:
            rc = lib.gen_fixed_indegree(inst.graph_seed, inst_index0 + b, inst.n, inst.n_exc, inst.k_exc, inst.k_inh, lo,
                                        ebase, ro_ptr, tg_ptr, threads)
            if rc != 0:
                raise ValueError(f"bad fixed in-degree recipe for instance {b}")
        lib.gen_fill_weights(row_off.ctypes.data + 8 * lo, inst.n, inst.n_exc, inst.w_exc_q, inst.w_inh_q,
                             w.ctypes.data)
        ebase += counts[b]
    assert int(row_off[N]) == E
    # every row carries its source population's weight (gen_fill_weights)
    w_row = np.zeros(N, dtype=np.int32)
    for b, inst in enumerate(prob.instances):
        lo = int(inst_off[b])
        w_row[lo:lo + inst.n_exc] = inst.w_exc_q
        w_row[lo + inst.n_exc:lo + inst.n] = inst.w_inh_q
    w_row[np.diff(row_off) == 0] = 0
    prob.inst_off, prob.row_off, prob.tgt, prob.w = inst_off, row_off, tgt, w
    prob._w_row, prob._w_row_of = w_row, w
    return prob


# ---------------------------------------------------------------------------
# Model recipes (Section IV: Vogels-Abbott, Brunel, Brunel with STDP)
# ---------------------------------------------------------------------------

def vogels_instance(n: int = 4000, *, k: int | None = None, p_conn: float = 0.02, c: float = 1.0,
                    graph_seed: int = 1) -> Instance:
    """Vogels-Abbott CUBA LIF: tau_m 20 ms, V_reset -60 mV, V_th -50 mV,
    E_L -49 mV (the standard CUBA benchmark's constant drive), 5 ms
    refractory, exponential currents tau_e 5 ms / tau_i 10 ms, weights
    1.62 / -9 mV scaled by c, V0 ~ U[-60, -50) mV, 80 % excitatory."""
    n_exc = (n * 4) // 5
    inst = Instance(n=n, n_exc=n_exc, dt=0.1, tau_m=20.0, v_th=-50.0, v_reset=-60.0, refractory_steps=50,
                    e_l=-49.0, tau_e=5.0, tau_i=10.0, v0_lo=-60.0, v0_span=10.0,
                    w_exc_mV=1.62 * c, w_inh_mV=-9.0 * c, graph_seed=graph_seed)
    if k is None:
        inst.p_conn = p_conn
    else:
        inst.k_exc = (k * 4) // 5
        inst.k_inh = k - inst.k_exc
    return inst


def brunel_instance(n: int = 12500, *, k: int = 1250, g: float = 5.0, nu_ratio: float = 2.0, J: float = 0.1,
                    graph_seed: int = 1, stdp: bool = False) -> Instance:
    """Brunel sparse network: tau 20 ms, theta 20 mV, V_r 10 mV, 2 ms
    refractory, J, -gJ, fixed in-degree k (80/20), external Poisson drive of
    nu_ext = nu_ratio * nu_thr over C_E inputs, i.e. lambda = nu_ratio *
    theta * dt / (J * tau) spikes of weight J per step."""
    n_exc = (n * 4) // 5
    k_exc = (k * 4) // 5
    theta, tau, dt = 20.0, 20.0, 0.1
    inst = Instance(n=n, n_exc=n_exc, dt=dt, tau_m=tau, v_th=theta, v_reset=10.0, refractory_steps=20,
                    lam=nu_ratio * theta * dt / (J * tau), jext_q=quantize_mV(J), v0_lo=0.0, v0_span=theta,
                    k_exc=k_exc, k_inh=k - k_exc, w_exc_mV=J, w_inh_mV=-g * J, graph_seed=graph_seed)
    if stdp:
        inst.tau_plus = 20.0
        inst.tau_minus = 20.0
        inst.a_plus = 0.01
        inst.a_minus = -0.0105
        inst.w_max_q = 2 * quantize_mV(J)
    return inst


def problem(model: int, instances: list, *, delay: int, n_steps: int, seed: int = 1, stdp: bool = False,
            threads: int | None = None, inst_index0: int = 0) -> Problem:
    return build_graph(Problem(model=model, instances=instances, delay=delay, seed=seed, n_steps=n_steps,
                               stdp=stdp), threads=threads, inst_index0=inst_index0)


def vogels_4k(seed: int = 1, n_steps: int = 1000) -> Problem:
    """Vogels-Abbott, 4,000 neurons, 2 % Bernoulli connectivity, no delay
    beyond the one-step minimum, 1,000 steps."""
    return problem(VOGELS, [vogels_instance(4000, graph_seed=seed)], delay=1, n_steps=n_steps, seed=seed)


def brunel_12k5(seed: int = 1, n_steps: int = 10000) -> Problem:
    """Brunel, 10,000 + 2,500 neurons, C_E 1,000 / C_I 250, g 5, 1.5 ms
    delay (15 steps), nu_ext = 2 nu_thr, 10,000 steps."""
    return problem(BRUNEL, [brunel_instance(12500, k=1250, graph_seed=seed)], delay=15, n_steps=n_steps,
                   seed=seed)


def vogels_1m(seed: int = 1, n_steps: int = 1000, n: int = 1_000_000, k: int = 1000) -> Problem:
    """Vogels-Abbott scaled to 1,000,000 neurons with fixed in-degree 1,000;
    weights scaled by c = 80 / 1000 to keep the mean input of the 4k net."""
    return problem(VOGELS, [vogels_instance(n, k=k, c=80.0 / k, graph_seed=seed)], delay=1, n_steps=n_steps,
                   seed=seed)


def brunel_stdp_100k(seed: int = 1, n_steps: int = 10000, n: int = 100_000, k: int = 1000) -> Problem:
    """Brunel+ : 100,000 neurons, in-degree 1,000, 15-step delay, additive
    pair STDP on exc->exc synapses clipped to [0, 2J]."""
    return problem(BRUNEL, [brunel_instance(n, k=k, graph_seed=seed, stdp=True)], delay=15, n_steps=n_steps,
                   seed=seed, stdp=True)


def batched_sweep_params(n_nets: int = 256, base_seed: int = 1, n_lo: int = 1000, n_hi: int = 50000,
                         k_cap: int = 1000) -> list:
    """The batched sweep: n_nets Brunel networks of log-uniform size in
    [n_lo, n_hi], in-degree 10 % capped at k_cap, g ~ U[3, 7],
    nu_ext / nu_thr ~ U[0.9, 4], graph seed base_seed + i."""
    rng = np.random.Generator(np.random.PCG64(base_seed))
    out = []
    for i in range(n_nets):
        n = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        k = min(int(math.ceil(0.1 * n)), k_cap)
        g = float(rng.uniform(3.0, 7.0))
        nu = float(rng.uniform(0.9, 4.0))
        out.append(brunel_instance(n, k=k, g=g, nu_ratio=nu, graph_seed=base_seed + i))
    return out


def batched_sweep(n_nets: int = 256, base_seed: int = 1, n_steps: int = 5000, threads: int | None = None,
                  **kw) -> Problem:
    return problem(BRUNEL, batched_sweep_params(n_nets, base_seed, **kw), delay=15, n_steps=n_steps,
                   seed=base_seed, threads=threads)


def sub_problem(prob: Problem, b: int, n_steps: int | None = None) -> Problem:
    """Instance b of a batch as a one-instance problem (ids rebased to 0)."""
    lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
    e0, e1 = int(prob.row_off[lo]), int(prob.row_off[hi])
    return Problem(model=prob.model, instances=[prob.instances[b]], delay=prob.delay, seed=prob.seed,
                   n_steps=prob.n_steps if n_steps is None else n_steps, stdp=prob.stdp,
                   inst_off=np.array([0, hi - lo], np.uint32),
                   row_off=(prob.row_off[lo:hi + 1] - np.uint64(e0)).astype(np.uint64),
                   tgt=(prob.tgt[e0:e1] - np.uint32(lo)).astype(np.uint32), w=prob.w[e0:e1].copy())


def from_edges(model: int, inst: Instance, edges, weights, *, delay: int, n_steps: int, seed: int = 1,
               stdp: bool = False) -> Problem:
    """A one-instance problem from an explicit edge list [(src, tgt)] and
    per-edge lattice weights (rows sorted by target)."""
    order = sorted(range(len(edges)), key=lambda k: edges[k])
    row_off = np.zeros(inst.n + 1, np.uint64)
    for s, _ in edges:
        row_off[s + 1] += 1
    row_off = np.cumsum(row_off).astype(np.uint64)
    tgt = np.array([edges[k][1] for k in order], np.uint32)
    w = np.array([weights[k] for k in order], np.int32)
    return Problem(model=model, instances=[inst], delay=delay, seed=seed, n_steps=n_steps, stdp=stdp,
                   inst_off=np.array([0, inst.n], np.uint32), row_off=row_off, tgt=tgt, w=w)
