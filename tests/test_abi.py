"""The C ABI library loads and exports every function include/*.h declares.

Runs without a GPU: it loads libsnn.so and makes only calls that fail on
their arguments before touching the device.
"""
import ctypes
import glob
import os
import re

import pytest

import paper_1912_07423_b300 as snn

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(snn_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_library_exports_every_declared_function():
    lib = snn.load()
    names = declared_functions()
    assert "snn_create" in names and "snn_step" in names and "snn_destroy" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(snn.exported_symbols()) <= set(names)


def test_argument_errors_without_device():
    lib = snn.load()
    ctx = ctypes.c_void_p()
    cfg = snn.Config(0, 0, 0, 1, 1, 0, 0, 0, 0, 0)  # delay 0 is invalid
    p = (snn.Params * 1)()
    p[0].n, p[0].n_exc, p[0].dt, p[0].tau_m, p[0].tau_e, p[0].tau_i = 10, 8, 0.1, 20.0, 5.0, 10.0
    assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    assert ctx.value is None
    cfg = snn.Config(0, snn.F_STDP, 1, 1, 1, 0, 0, 0, 0, 0)  # STDP needs the Brunel model
    assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    cfg = snn.Config(1, snn.F_LAZY, 1, 1, 1, 0, 0, 0, 0, 0)  # lazy plasticity needs STDP
    assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    for fifo in (1, 129):  # the history is 2..128 steps
        cfg = snn.Config(1, snn.F_STDP | snn.F_LAZY, 1, 1, 1, 0, 0, 0, 0, fifo)
        assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    cfg = snn.Config(1, 0, 1, 1, 1, 0, 0, 0, 0, 0)
    p[0].lam = 500.0  # Poisson table would exceed 64 entries
    assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    p[0].lam = 2.0
    p[0].refractory_steps = 300
    assert lib.snn_create(ctypes.byref(cfg), ctypes.addressof(p), None, ctypes.byref(ctx)) == -1
    assert lib.snn_create(None, None, None, ctypes.byref(ctx)) == -1
    # NULL-safe calls
    lib.snn_destroy(None)
    assert lib.snn_step(None, 1) == -1
    assert lib.snn_build_graph(None, None, None, None) == -1
    assert lib.snn_build_graph_rows(None, None, None, None) == -1
    assert lib.snn_last_error(None) == b""
    assert lib.snn_status_string(-4) == b"overflow"


def test_no_cpu_fallback_without_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    import snn_inputs as si
    prob = si.vogels_4k(n_steps=10)
    with pytest.raises(snn.SnnError):
        snn.Network(prob)
