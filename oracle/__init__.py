"""CPU oracle of the work-queue SNN timestep -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product (``paper_1912_07423_b300``)
never imports it and shares no code with it.

The simulation itself is plain C (``snn_oracle.c``): a slow, single-threaded,
eager clock-driven simulator written from the paper's pipeline
(Section III-A-1, Fig. 1).  This wrapper only marshals arguments.

Parity status of the functions (what pins each one, see tests/test_oracle_*):
  philox      -- numpy's Philox4x64-10 bit generator (library routine)
  poisson     -- scipy.stats.poisson CDF and sample moments / chi-square
  run (f32)   -- LIF closed forms, exact d-step FIFO arrival, the relay
                 (ping-pong) network against breadth-first search, a dense
                 matrix brute force of Receive Spikes, closed-form STDP
                 weight changes of a single pre/post pair, the Init stage's
                 V0 draw against numpy's Philox words and the uniform law on
                 [v0_lo, v0_lo + v0_span), the Brunel refractory clamp (period
                 R + 1 under forced drive; input inside the clamp discarded)
  run_f64     -- agreement with the binary32 run in population rate and
                 ISI CV (statistical; it is a comparison variant)
  relay_raster -- a hand-worked raster of a four-neuron graph, breadth-first
                 search over the CSR, and the binary32 run of the same graph
                 in its LIF relay form
  expand_jobs -- Fig. 2's printed spacings, running sums and normalised
                 values, the binary64 library logarithm, the exact law of
                 each rounded order statistic, full and empty ranges
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = [os.path.join(_HERE, "snn_oracle.c"), os.path.join(_HERE, "snn_oracle.h")]
_SO = os.path.join(_HERE, "libsnn_oracle.so")
_lock = threading.Lock()
_lib = None

POISSON_CAP = 64
CFLAGS = ["-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-msse2",
          "-mfpmath=sse", "-fexcess-precision=standard"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc.  Building the checker is not using it."""
    newest = max(os.path.getmtime(p) for p in _SRC)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < newest:
        subprocess.check_call(["gcc", *CFLAGS, "-o", _SO + ".tmp", _SRC[0], "-lm"])
        os.replace(_SO + ".tmp", _SO)
    return _SO


class _Params(ctypes.Structure):
    _fields_ = [("n_exc", ctypes.c_uint32), ("refractory_steps", ctypes.c_uint32), ("jext_q", ctypes.c_int32),
                ("w_max_q", ctypes.c_int32), ("dt", ctypes.c_double), ("tau_m", ctypes.c_double),
                ("v_th", ctypes.c_double), ("v_reset", ctypes.c_double), ("e_l", ctypes.c_double),
                ("tau_e", ctypes.c_double), ("tau_i", ctypes.c_double), ("lam", ctypes.c_double),
                ("v0_lo", ctypes.c_double), ("v0_span", ctypes.c_double), ("tau_plus", ctypes.c_double),
                ("tau_minus", ctypes.c_double), ("a_plus", ctypes.c_double), ("a_minus", ctypes.c_double)]


_vp = ctypes.c_void_p


class _Problem(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int32), ("stdp", ctypes.c_int32), ("n_inst", ctypes.c_uint32),
                ("delay", ctypes.c_uint32), ("inst_off", _vp), ("params", _vp), ("seed", ctypes.c_uint64),
                ("row_off", _vp), ("tgt", _vp), ("w", _vp), ("n_steps", ctypes.c_uint32),
                ("n_over", ctypes.c_uint32), ("over_step", _vp), ("over_id", _vp), ("over_v", _vp),
                ("inst_key0", ctypes.c_uint32), ("pad", ctypes.c_uint32)]


class _State(ctypes.Structure):
    _fields_ = [("init_given", ctypes.c_int32), ("V", _vp), ("ge", _vp), ("gi", _vp), ("r", _vp), ("x", _vp),
                ("y", _vp), ("acc0", _vp), ("acc1", _vp), ("w", _vp)]


class _Raster(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("step", ctypes.POINTER(ctypes.c_uint32)),
                ("id", ctypes.POINTER(ctypes.c_uint32)), ("events", ctypes.c_uint64)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_philox4x64_10.argtypes = [_vp, _vp, _vp]
            lib.orc_philox4x64_10.restype = None
            lib.orc_rand_word.argtypes = [ctypes.c_uint64] * 5
            lib.orc_rand_word.restype = ctypes.c_uint32
            lib.orc_poisson_table.argtypes = [ctypes.c_double, _vp, ctypes.c_int]
            lib.orc_poisson_table.restype = ctypes.c_int
            lib.orc_poisson_sample.argtypes = [_vp, ctypes.c_int, ctypes.c_uint32]
            lib.orc_poisson_sample.restype = ctypes.c_uint32
            lib.orc_receive.argtypes = [ctypes.POINTER(_Problem), _vp, _vp, ctypes.c_uint64, _vp, _vp, _vp]
            lib.orc_receive.restype = ctypes.c_int
            lib.orc_run.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_State), ctypes.POINTER(_Raster)]
            lib.orc_run.restype = ctypes.c_int
            lib.orc_run_f64.argtypes = [ctypes.POINTER(_Problem), _vp, _vp, ctypes.POINTER(_Raster)]
            lib.orc_run_f64.restype = ctypes.c_int
            lib.orc_raster_free.argtypes = [ctypes.POINTER(_Raster)]
            lib.orc_raster_free.restype = None
            lib.orc_neg_ln.argtypes = [ctypes.c_float]
            lib.orc_neg_ln.restype = ctypes.c_float
            lib.orc_job_from_uniforms.argtypes = [_vp, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, _vp]
            lib.orc_job_from_uniforms.restype = ctypes.c_int
            lib.orc_expand_jobs.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp, ctypes.c_uint64]
            lib.orc_expand_jobs.restype = ctypes.c_int
            lib.orc_expand_job.argtypes = [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp]
            lib.orc_expand_job.restype = ctypes.c_int
            _lib = lib
    return _lib


class OracleError(RuntimeError):
    pass


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a is not None and a.size else 0


def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block."""
    c = np.ascontiguousarray(ctr, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def rand_word(seed: int, inst: int, local: int, step: int, tag: int) -> int:
    return int(_load().orc_rand_word(seed, inst, local, step, tag))


# a job of the adjacency construction (Fig. 2): n, a, b, reserved, o
JOB_DTYPE = np.dtype([("n", "<u4"), ("a", "<u4"), ("b", "<u4"), ("reserved", "<u4"), ("o", "<u8")])


def neg_ln(u: float) -> float:
    """-ln(u), u in (0, 1], the oracle's own binary32 logarithm (Fig. 2)."""
    return float(_load().orc_neg_ln(ctypes.c_float(u)))


def job_from_uniforms(u, a: int, b: int):
    """The steps of one job (Fig. 2) from its uniforms u[0..n]: returns
    (q, c, out) -- integer spacings, exclusive running sums (c[n+1] is the
    total) and the n output values."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    n = u.size - 1
    q = np.zeros(n + 1, dtype=np.uint32)
    c = np.zeros(n + 2, dtype=np.uint64)
    out = np.zeros(max(n, 1), dtype=np.uint32)
    st = _load().orc_job_from_uniforms(_ptr(u), n, a, b, _ptr(q), _ptr(c), _ptr(out))
    if st != 0:
        raise OracleError(f"job_from_uniforms failed ({st})")
    return q, c, out[:n]


def expand_jobs(jobs: np.ndarray, seed: int, out_len: int) -> np.ndarray:
    """Expand jobs (JOB_DTYPE records) into a uint32 array of out_len values;
    entries no job writes stay 0xffffffff."""
    jobs = np.ascontiguousarray(jobs, dtype=JOB_DTYPE)
    out = np.full(max(out_len, 1), 0xffffffff, dtype=np.uint32)
    st = _load().orc_expand_jobs(_ptr(jobs), jobs.size, seed, _ptr(out), out_len)
    if st != 0:
        raise OracleError(f"expand_jobs failed ({st})")
    return out[:out_len]


def expand_job(job, index: int, seed: int) -> np.ndarray:
    """One job (a JOB_DTYPE record) alone, by its index in the job list
    (which keys its random draws): its n values."""
    rec = np.ascontiguousarray(np.asarray(job, dtype=JOB_DTYPE).reshape(1))
    out = np.zeros(max(int(rec["n"][0]), 1), dtype=np.uint32)
    st = _load().orc_expand_job(_ptr(rec), index, seed, _ptr(out))
    if st != 0:
        raise OracleError(f"expand_job failed ({st})")
    return out[:int(rec["n"][0])]


def poisson_table(lam: float) -> np.ndarray:
    T = np.zeros(POISSON_CAP, dtype=np.uint32)
    n = _load().orc_poisson_table(lam, _ptr(T), POISSON_CAP)
    if n < 0:
        raise OracleError(f"poisson table failed ({n})")
    return T[:n].copy()


def poisson_sample(T: np.ndarray, u: int) -> int:
    T = np.ascontiguousarray(T, dtype=np.uint32)
    return int(_load().orc_poisson_sample(_ptr(T), len(T), u))


class _Marshalled:
    """Keeps the numpy buffers alive while C holds pointers into them."""

    def __init__(self, prob, overrides=None, inst_key0=0):
        B = len(prob.instances)
        self.params = (_Params * B)()
        for b, inst in enumerate(prob.instances):
            p = self.params[b]
            p.n_exc, p.refractory_steps = inst.n_exc, inst.refractory_steps
            p.jext_q, p.w_max_q = inst.jext_q, inst.w_max_q
            p.dt, p.tau_m, p.v_th, p.v_reset = inst.dt, inst.tau_m, inst.v_th, inst.v_reset
            p.e_l, p.tau_e, p.tau_i, p.lam = inst.e_l, inst.tau_e, inst.tau_i, inst.lam
            p.v0_lo, p.v0_span = inst.v0_lo, inst.v0_span
            p.tau_plus, p.tau_minus, p.a_plus, p.a_minus = inst.tau_plus, inst.tau_minus, inst.a_plus, inst.a_minus
        self.inst_off = np.ascontiguousarray(prob.inst_off, dtype=np.uint32)
        self.row_off = np.ascontiguousarray(prob.row_off, dtype=np.uint64)
        self.tgt = np.ascontiguousarray(prob.tgt, dtype=np.uint32)
        self.w = np.ascontiguousarray(prob.w, dtype=np.int32)
        ov = sorted(overrides or [], key=lambda o: o[0])
        self.over_step = np.array([o[0] for o in ov], dtype=np.uint32)
        self.over_id = np.array([o[1] for o in ov], dtype=np.uint32)
        self.over_v = np.array([o[2] for o in ov], dtype=np.float32)
        P = _Problem()
        P.model, P.stdp, P.n_inst, P.delay = prob.model, int(bool(prob.stdp)), B, prob.delay
        P.inst_off, P.params, P.seed = _ptr(self.inst_off), ctypes.addressof(self.params), prob.seed
        P.row_off, P.tgt, P.w, P.n_steps = _ptr(self.row_off), _ptr(self.tgt), _ptr(self.w), prob.n_steps
        P.n_over = len(ov)
        P.over_step, P.over_id, P.over_v = _ptr(self.over_step), _ptr(self.over_id), _ptr(self.over_v)
        P.inst_key0 = inst_key0
        self.P = P


def _take_raster(lib, R):
    n = int(R.n)
    steps = np.ctypeslib.as_array(R.step, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
    ids = np.ctypeslib.as_array(R.id, shape=(n,)).copy() if n else np.zeros(0, np.uint32)
    lib.orc_raster_free(ctypes.byref(R))
    return steps, ids


def run(prob, overrides=None, state=None, inst_key0: int = 0) -> dict:
    """Simulate prob.n_steps steps in binary32.

    overrides: list of (step, neuron, V) applied before that step's update.
    state: optional dict of initial arrays (V, ge, gi, r, x, y, acc0, acc1,
    w); default draws N_0 as documented in snn_oracle.c.
    inst_key0: Philox instance key of the problem's first instance (to re-run
    instance b of a batch alone, pass a one-instance problem and b).
    Returns the raster (steps, ids sorted by (step, id)), the delivered event
    count and the final state."""
    lib = _load()
    m = _Marshalled(prob, overrides, inst_key0)
    N, E = prob.n, prob.n_edges
    st = {
        "V": np.zeros(N, np.float32), "ge": np.zeros(N, np.float32), "gi": np.zeros(N, np.float32),
        "r": np.zeros(N, np.int32), "x": np.zeros(N, np.float32), "y": np.zeros(N, np.float32),
        "acc0": np.zeros(N, np.int32), "acc1": np.zeros(N, np.int32), "w": np.zeros(max(E, 1), np.int32)[:E],
    }
    S = _State()
    S.init_given = 0
    if state is not None:
        S.init_given = 1
        for k, v in state.items():
            st[k][...] = v
    for k in ("V", "ge", "gi", "r", "x", "y", "acc0", "acc1", "w"):
        setattr(S, k, _ptr(st[k]))
    R = _Raster()
    rc = lib.orc_run(ctypes.byref(m.P), ctypes.byref(S), ctypes.byref(R))
    if rc != 0:
        lib.orc_raster_free(ctypes.byref(R))
        raise OracleError(f"orc_run failed ({rc})")
    steps, ids = _take_raster(lib, R)
    out = dict(st)
    out.update(steps=steps, ids=ids, events=int(R.events))
    return out


def run_f64(prob, w_mV: np.ndarray | None = None, inst_key0: int = 0) -> dict:
    """The binary64, unquantised-weight comparison variant (no STDP).
    inst_key0 as for run()."""
    lib = _load()
    m = _Marshalled(prob, inst_key0=inst_key0)
    wd = np.ascontiguousarray(prob.w_mV() if w_mV is None else w_mV, dtype=np.float64)
    V = np.zeros(prob.n, np.float64)
    R = _Raster()
    rc = lib.orc_run_f64(ctypes.byref(m.P), _ptr(wd), _ptr(V), ctypes.byref(R))
    if rc != 0:
        lib.orc_raster_free(ctypes.byref(R))
        raise OracleError(f"orc_run_f64 failed ({rc})")
    steps, ids = _take_raster(lib, R)
    return {"steps": steps, "ids": ids, "events": int(R.events), "V": V}


def receive(prob, spikes, w=None) -> tuple:
    """Receive Spikes alone: deliver the given spike ids along their rows
    into fresh int64 accumulators (channel 0 and channel 1)."""
    lib = _load()
    m = _Marshalled(prob)
    sp = np.ascontiguousarray(spikes, dtype=np.uint32)
    wa = m.w if w is None else np.ascontiguousarray(w, dtype=np.int32)
    acc0 = np.zeros(prob.n, np.int64)
    acc1 = np.zeros(prob.n, np.int64)
    ev = ctypes.c_uint64(0)
    rc = lib.orc_receive(ctypes.byref(m.P), _ptr(wa), _ptr(sp), len(sp), _ptr(acc0), _ptr(acc1),
                         ctypes.addressof(ev))
    if rc != 0:
        raise OracleError(f"orc_receive failed ({rc})")
    return acc0, acc1, int(ev.value)


def relay_raster(prob, n_steps: int | None = None) -> dict:
    """The tutorial model of Section III-B (Listing 1), written from its
    definition with plain loops: every neuron holds a flag, set before step
    0 for the first population of its instance (local id < n_exc); at each
    step a neuron fires when its flag is set or the lattice weights it
    received since its previous update sum to a nonzero value, and the flag
    clears.  A spike of step t is delivered along its row at step t + d - 1
    and so reaches the update of step t + d (the delay FIFO of Fig. 1).
    Returns the raster sorted by (step, id), the events delivered within the
    run, and the input pending for the next update (acc0)."""
    T = prob.n_steps if n_steps is None else n_steps
    d = int(prob.delay)
    n = int(prob.n)
    inst_off = [int(v) for v in prob.inst_off]
    row_off = [int(v) for v in prob.row_off]
    tgt = [int(v) for v in prob.tgt]
    w = [int(v) for v in prob.w]
    flag = [0] * n
    for b, inst in enumerate(prob.instances):
        for local in range(min(inst.n_exc, inst.n)):
            flag[inst_off[b] + local] = 1
    arrive = {}  # step -> {neuron: summed weight}
    steps, ids, events = [], [], 0
    for t in range(T):
        got = arrive.pop(t, {})
        fired = []
        for i in range(n):
            if flag[i] or got.get(i, 0) != 0:
                fired.append(i)
            flag[i] = 0
        for i in fired:
            steps.append(t)
            ids.append(i)
        if t + d - 1 <= T - 1:  # delivered inside the run
            into = arrive.setdefault(t + d, {})
            for j in fired:
                for e in range(row_off[j], row_off[j + 1]):
                    into[tgt[e]] = into.get(tgt[e], 0) + w[e]
                events += row_off[j + 1] - row_off[j]
    acc0 = np.zeros(n, np.int64)
    for i, v in arrive.get(T, {}).items():
        acc0[i] = v
    return {"steps": np.array(steps, np.uint32), "ids": np.array(ids, np.uint32), "events": events, "acc0": acc0}
