"""B300-native work-queue SNN timestep: Python binding of libsnn (include/snn.h).

Argument marshalling only.  Every step of the simulation runs in the CUDA
kernels of ``csrc/``; PyTorch provides the device memory (its caching
allocator, through the library's allocation callbacks) and the stream.
There is no CPU fallback: without the compiled library or a CUDA device the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .build import LIB, build as _build

__all__ = ["Network", "SnnError", "load", "VOGELS", "BRUNEL", "MODEL_RELAY", "MODEL_BRUNEL_LIF", "MODEL_STATE_DTYPE",
           "RECV_AUTO", "RECV_GLOBAL", "RECV_TILED", "RECV_BULK", "RECV_PERSISTENT", "F_STDP", "F_W16", "F_STATS", "F_UNPACKED", "F_LAZY",
           "F_SERIAL", "FIELDS"]

VOGELS, BRUNEL = 0, 1
# models of the generic update (snn_models.cuh) and their per-neuron state records
MODEL_RELAY, MODEL_BRUNEL_LIF = 2, 3
MODEL_STATE_DTYPE = {
    MODEL_RELAY: np.dtype([("flag", "u1")]),
    MODEL_BRUNEL_LIF: np.dtype({"names": ["V", "r"], "formats": ["<f4", "u1"], "offsets": [0, 4], "itemsize": 8}),
}
F_STDP, F_W16, F_STATS, F_UNPACKED, F_LAZY, F_SERIAL = 1, 2, 4, 8, 16, 32
RECV_AUTO, RECV_GLOBAL, RECV_TILED, RECV_BULK, RECV_PERSISTENT = 0, 1, 2, 3, 4
FIELDS = {"V": 0, "ge": 1, "gi": 2, "r": 3, "x": 4, "y": 5, "acc0": 6, "acc1": 7, "w": 8, "model": 9}
_FIELD_DTYPE = {"V": np.float32, "ge": np.float32, "gi": np.float32, "r": np.int32, "x": np.float32,
                "y": np.float32, "acc0": np.int32, "acc1": np.int32, "w": np.int32}

_vp = ctypes.c_void_p
_lock = threading.Lock()
_lib = None


class SnnError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"libsnn status {status}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    _fields_ = [("model", ctypes.c_uint32), ("flags", ctypes.c_uint32), ("delay", ctypes.c_uint32),
                ("n_inst", ctypes.c_uint32), ("seed", ctypes.c_uint64), ("log_capacity", ctypes.c_uint64),
                ("receive", ctypes.c_uint32), ("steps_per_graph", ctypes.c_uint32), ("tune_steps", ctypes.c_uint32),
                ("lazy_fifo", ctypes.c_uint32), ("wait_polls", ctypes.c_uint32), ("inst_key0", ctypes.c_uint32)]


class Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("n_exc", ctypes.c_uint32), ("refractory_steps", ctypes.c_uint32),
                ("jext_q", ctypes.c_int32), ("w_max_q", ctypes.c_int32), ("reserved", ctypes.c_uint32),
                ("dt", ctypes.c_double), ("tau_m", ctypes.c_double), ("v_th", ctypes.c_double),
                ("v_reset", ctypes.c_double), ("e_l", ctypes.c_double), ("tau_e", ctypes.c_double),
                ("tau_i", ctypes.c_double), ("lam", ctypes.c_double), ("v0_lo", ctypes.c_double),
                ("v0_span", ctypes.c_double), ("tau_plus", ctypes.c_double), ("tau_minus", ctypes.c_double),
                ("a_plus", ctypes.c_double), ("a_minus", ctypes.c_double)]


class Info(ctypes.Structure):
    _fields_ = [("receive", ctypes.c_uint32), ("n_tiles", ctypes.c_uint32), ("n_padded", ctypes.c_uint32),
                ("rows_sorted", ctypes.c_uint32), ("edges", ctypes.c_uint64), ("device_bytes", ctypes.c_uint64),
                ("edge_bytes", ctypes.c_uint32), ("model_state_bytes", ctypes.c_uint32), ("fused", ctypes.c_uint32),
                ("tuned", ctypes.c_uint32), ("tune_ms", ctypes.c_float * 5), ("persistent", ctypes.c_uint32),
                ("persist_ctas", ctypes.c_uint32)]


ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, _vp, _vp)


class Device(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("user", _vp), ("stream", _vp)]


def load():
    """Load libsnn.so (building it first if its sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = LIB if os.path.exists(LIB) and os.environ.get("SNN_NO_BUILD") else _build()
            lib = ctypes.CDLL(path)
            S = ctypes.c_int
            sigs = {
                "snn_create": (S, [ctypes.POINTER(Config), _vp, ctypes.POINTER(Device), ctypes.POINTER(_vp)]),
                "snn_build_graph": (S, [_vp, _vp, _vp, _vp]),
                "snn_build_graph_rows": (S, [_vp, _vp, _vp, _vp]),
                "snn_reset": (S, [_vp]),
                "snn_step": (S, [_vp, ctypes.c_uint32]),
                "snn_sync": (S, [_vp]),
                "snn_step_profiled": (S, [_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double)]),
                "snn_read_spikes": (S, [_vp, ctypes.c_uint32, ctypes.c_uint32, _vp, _vp, ctypes.c_uint64,
                                        ctypes.POINTER(ctypes.c_uint64)]),
                "snn_log_clear": (S, [_vp]),
                "snn_read_state": (S, [_vp, ctypes.c_int, _vp]),
                "snn_write_state": (S, [_vp, ctypes.c_int, _vp]),
                "snn_counters": (S, [_vp, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_uint64),
                                     ctypes.POINTER(ctypes.c_uint64)]),
                "snn_stats": (S, [_vp, ctypes.c_uint32, ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
                "snn_stats_clear": (S, [_vp]),
                "snn_get_info": (S, [_vp, ctypes.POINTER(Info)]),
                "snn_rate_cv_static": (S, [_vp, _vp, _vp, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, _vp,
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
                "snn_expand_jobs": (S, [_vp, ctypes.c_uint64, ctypes.c_uint64, _vp, ctypes.c_uint64, _vp]),
                "snn_last_error": (ctypes.c_char_p, [_vp]),
                "snn_status_string": (ctypes.c_char_p, [ctypes.c_int]),
                "snn_destroy": (None, [_vp]),
            }
            for name, (res, args) in sigs.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def exported_symbols() -> list:
    return ["snn_create", "snn_build_graph", "snn_build_graph_rows", "snn_reset", "snn_step", "snn_step_profiled", "snn_sync",
            "snn_read_spikes",
            "snn_log_clear", "snn_read_state", "snn_write_state", "snn_counters", "snn_stats", "snn_stats_clear",
            "snn_get_info", "snn_rate_cv_static", "snn_expand_jobs", "snn_last_error", "snn_status_string",
            "snn_destroy"]


# a job of the adjacency construction (snn_job): n, a, b, reserved, o
JOB_DTYPE = np.dtype([("n", "<u4"), ("a", "<u4"), ("b", "<u4"), ("reserved", "<u4"), ("o", "<u8")])


def expand_jobs(jobs, seed: int, out_len: int, *, out=None, device: str = "cuda:0", stream=None):
    """Adjacency construction on the GPU (snn_expand_jobs, Fig. 2).  jobs: a
    JOB_DTYPE array (host) or a uint8 CUDA tensor of such records; returns
    the uint32 values as an int32 CUDA tensor of out_len elements (out, if
    given, is written instead; slots no job writes keep their contents)."""
    import torch
    if not torch.cuda.is_available():
        raise SnnError(-3, "no CUDA device: libsnn has no CPU fallback")
    lib = load()
    dev = torch.device(device)
    if isinstance(jobs, np.ndarray):
        jobs = np.ascontiguousarray(jobs, dtype=JOB_DTYPE)
        n_jobs = jobs.size
        djobs = torch.from_numpy(jobs.view(np.uint8)).to(dev)
    else:
        djobs = jobs
        n_jobs = djobs.numel() // JOB_DTYPE.itemsize
    if out is None:
        out = torch.empty(max(out_len, 1), dtype=torch.int32, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    rc = lib.snn_expand_jobs(djobs.data_ptr() if n_jobs else None, n_jobs, seed, out.data_ptr(), out_len,
                             st.cuda_stream)
    if rc != 0:
        raise SnnError(rc, "snn_expand_jobs: " + lib.snn_status_string(rc).decode())
    return out[:out_len]


def _params_array(instances) -> ctypes.Array:
    arr = (Params * len(instances))()
    for b, inst in enumerate(instances):
        p = arr[b]
        p.n, p.n_exc, p.refractory_steps = inst.n, inst.n_exc, inst.refractory_steps
        p.jext_q, p.w_max_q = inst.jext_q, inst.w_max_q
        p.dt, p.tau_m, p.v_th, p.v_reset = inst.dt, inst.tau_m, inst.v_th, inst.v_reset
        p.e_l, p.tau_e, p.tau_i, p.lam = inst.e_l, inst.tau_e, inst.tau_i, inst.lam
        p.v0_lo, p.v0_span = inst.v0_lo, inst.v0_span
        p.tau_plus, p.tau_minus, p.a_plus, p.a_minus = inst.tau_plus, inst.tau_minus, inst.a_plus, inst.a_minus
    return arr


class _TorchMemory:
    """Device memory from torch's caching allocator, on the given stream."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.live = {}
        self.alloc_cb = ALLOC_FN(self._alloc)
        self.free_cb = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, user):
        try:
            t = self.torch.empty(int(nbytes), dtype=self.torch.uint8, device=self.device)
        except Exception:
            return None
        ptr = t.data_ptr()
        self.live[ptr] = t
        return ptr

    def _free(self, ptr, stream, user):
        self.live.pop(ptr, None)


class Network:
    """One simulator context: many network instances stepped together.

    problem: an ``snn_inputs.Problem`` (model, instances, delay, seed, graph);
    its model may be VOGELS, BRUNEL or a generic-update model (MODEL_RELAY,
    MODEL_BRUNEL_LIF), whose state records ``read("model")`` returns.
    w16: 16-bit weight codes (else binary32).  receive: RECV_*.
    log_capacity: raster-log entries (default 64 per neuron, at least 65,536),
    shared out among the instances in proportion to their neurons.
    packed: let the receives read compressed edges (row weights, 16-bit
    target offsets, packed offset + code) where they can.
    lazy, lazy_fifo: with STDP, the lazy Update Synapses and its history
    length in steps (0: 128).  stats: keep spike counts and ISI moments.
    wait_polls: bound of the bulk receive's mbarrier waits and of the
    persistent launch's grid barrier (0: the defaults).
    inst_key0: Philox instance key of the first instance (to re-run network b
    of a batch alone with its own random numbers, pass b).
    serial: run Update Neurons and Receive Spikes as separate kernels even
    where the fused step applies.
    steps_per_graph, tune_steps: CUDA-graph length and bulk re-plan step.
    build_graph: upload problem's graph now (else call build_graph).
    Every call goes through the C ABI; there is no CPU path.
    """

    def __init__(self, problem, *, w16: bool = True, receive: int = RECV_AUTO, log_capacity: int | None = None,
                 stats: bool = False, steps_per_graph: int = 0, tune_steps: int = 0, device: str = "cuda:0",
                 stream=None, build_graph: bool = True, packed: bool = True, lazy: bool = False,
                 lazy_fifo: int = 0, wait_polls: int = 0, inst_key0: int = 0, serial: bool = False):
        import torch
        if not torch.cuda.is_available():
            raise SnnError(-3, "no CUDA device: libsnn has no CPU fallback")
        self.lib = load()
        self.problem = problem
        self.device = torch.device(device)
        torch.cuda.set_device(self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.mem = _TorchMemory(self.device)
        self.dev = Device(self.mem.alloc_cb, self.mem.free_cb, None, self.stream.cuda_stream)
        flags = (F_STDP if problem.stdp else 0) | (F_W16 if w16 else 0) | (F_STATS if stats else 0) | \
            (0 if packed else F_UNPACKED) | (F_LAZY if lazy else 0) | (F_SERIAL if serial else 0)
        if log_capacity is None:
            log_capacity = max(1 << 16, int(problem.n) * 64)
        self.cfg = Config(problem.model, flags, problem.delay, len(problem.instances), problem.seed, log_capacity,
                          receive, steps_per_graph, tune_steps, lazy_fifo, wait_polls, inst_key0)
        self.params = _params_array(problem.instances)
        ctx = _vp()
        st = self.lib.snn_create(ctypes.byref(self.cfg), ctypes.addressof(self.params), ctypes.byref(self.dev),
                                 ctypes.byref(ctx))
        if st != 0:
            raise SnnError(st, "snn_create failed: " + self.lib.snn_status_string(st).decode())
        self.ctx = ctx
        self.n = int(problem.inst_off[-1]) if problem.inst_off is not None else sum(i.n for i in problem.instances)
        if build_graph:
            w_row = problem.row_weights() if hasattr(problem, "row_weights") else None
            if w_row is not None:
                self.build_graph_rows(problem.row_off, problem.tgt, w_row)
            else:
                self.build_graph(problem.row_off, problem.tgt, problem.w)

    # -- plumbing -----------------------------------------------------------
    def _check(self, st: int, what: str):
        if st != 0:
            msg = self.lib.snn_last_error(self.ctx).decode()
            raise SnnError(st, f"{what}: {msg}")

    def close(self):
        if getattr(self, "ctx", None):
            self.lib.snn_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- API ----------------------------------------------------------------
    def build_graph(self, row_off, tgt, w_q):
        ro = np.ascontiguousarray(row_off, dtype=np.uint64)
        tg = np.ascontiguousarray(tgt, dtype=np.uint32)
        wq = np.ascontiguousarray(w_q, dtype=np.int32)
        self.n_edges = int(ro[-1])
        self._check(self.lib.snn_build_graph(self.ctx, ro.ctypes.data, tg.ctypes.data if tg.size else None,
                                             wq.ctypes.data if wq.size else None), "snn_build_graph")

    def build_graph_rows(self, row_off, tgt, w_row):
        """build_graph for rows that each carry one weight: w_row[j] for every
        synapse of row j (only the targets and one weight per row are copied)."""
        ro = np.ascontiguousarray(row_off, dtype=np.uint64)
        tg = np.ascontiguousarray(tgt, dtype=np.uint32)
        wr = np.ascontiguousarray(w_row, dtype=np.int32)
        self.n_edges = int(ro[-1])
        self._check(self.lib.snn_build_graph_rows(self.ctx, ro.ctypes.data, tg.ctypes.data if tg.size else None,
                                                  wr.ctypes.data if wr.size else None), "snn_build_graph_rows")

    def reset(self):
        self._check(self.lib.snn_reset(self.ctx), "snn_reset")

    def step(self, n_steps: int = 1):
        self._check(self.lib.snn_step(self.ctx, int(n_steps)), "snn_step")

    def step_profiled(self, n_steps: int) -> dict:
        """Steps with per-kernel CUDA events; summed device ms per phase."""
        ms = (ctypes.c_double * 6)()
        self._check(self.lib.snn_step_profiled(self.ctx, int(n_steps), ms), "snn_step_profiled")
        return dict(zip(["depress", "update", "potentiate", "receive", "merge", "step_end"], list(ms)))

    def sync(self):
        self._check(self.lib.snn_sync(self.ctx), "snn_sync")

    def spikes(self, t0: int = 0, t1: int = 2**32 - 1):
        """(steps, ids) of the logged spikes in [t0, t1), sorted by (step, id)."""
        n = ctypes.c_uint64(0)
        self._check(self.lib.snn_read_spikes(self.ctx, t0, t1, None, None, 0, ctypes.byref(n)), "snn_read_spikes")
        cnt = int(n.value)
        steps = np.zeros(max(cnt, 1), np.uint32)
        ids = np.zeros(max(cnt, 1), np.uint32)
        self._check(self.lib.snn_read_spikes(self.ctx, t0, t1, steps.ctypes.data, ids.ctypes.data, cnt,
                                             ctypes.byref(n)), "snn_read_spikes")
        return steps[:cnt], ids[:cnt]

    def log_clear(self):
        self._check(self.lib.snn_log_clear(self.ctx), "snn_log_clear")

    def _dtype(self, field: str):
        if field == "model":
            if self.problem.model not in MODEL_STATE_DTYPE:
                raise SnnError(-1, "the model field exists for the generic models only")
            return MODEL_STATE_DTYPE[self.problem.model]
        return _FIELD_DTYPE[field]

    def read(self, field: str) -> np.ndarray:
        size = self.n_edges if field == "w" else self.n
        out = np.zeros(max(size, 1), self._dtype(field))
        self._check(self.lib.snn_read_state(self.ctx, FIELDS[field], out.ctypes.data), f"snn_read_state({field})")
        return out[:size]

    def write(self, field: str, values):
        size = self.n_edges if field == "w" else self.n
        arr = np.ascontiguousarray(values, dtype=self._dtype(field))
        if arr.size != size:
            raise ValueError(f"{field}: expected {size} values, got {arr.size}")
        buf = arr if arr.size else np.zeros(1, arr.dtype)
        self._check(self.lib.snn_write_state(self.ctx, FIELDS[field], buf.ctypes.data), f"snn_write_state({field})")

    def counters(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        self._check(self.lib.snn_counters(self.ctx, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
                    "snn_counters")
        return {"steps": int(a.value), "spikes": int(b.value), "events": int(c.value)}

    def stats(self, inst: int = 0):
        r, cv = ctypes.c_double(), ctypes.c_double()
        self._check(self.lib.snn_stats(self.ctx, inst, ctypes.byref(r), ctypes.byref(cv)), "snn_stats")
        return float(r.value), float(cv.value)

    def stats_clear(self):
        self._check(self.lib.snn_stats_clear(self.ctx), "snn_stats_clear")

    def info(self) -> dict:
        i = Info()
        self._check(self.lib.snn_get_info(self.ctx, ctypes.byref(i)), "snn_get_info")
        return {"receive": {RECV_GLOBAL: "global", RECV_TILED: "tiled", RECV_BULK: "bulk"}.get(i.receive, "?"), "n_tiles": i.n_tiles,
                "n_padded": i.n_padded, "rows_sorted": bool(i.rows_sorted), "edges": i.edges,
                "device_bytes": i.device_bytes, "edge_bytes": i.edge_bytes, "model_state_bytes": i.model_state_bytes,
                "fused": bool(i.fused), "tuned": bool(i.tuned),
                "tune_ms": dict(zip(["global", "tiled", "fused", "bulk", "persistent"], [float(x) for x in i.tune_ms])),
                "persistent": bool(i.persistent), "persist_ctas": int(i.persist_ctas)}
