"""snn_rate_cv_static: rate and ISI CV for callers that cannot allocate.

Some applications hand all of the GPU's memory to their own arena at
start-up, or run latency-critical loops where a cudaMalloc could stall the
device; they cannot let the library allocate scratch when they ask for the
network statistics.  snn_rate_cv_static works from a fixed device array
inside the library instead.  Through the C ABI, on two calls in a row, its
results must equal those of snn_stats (which takes its scratch from the
allocator) on the same spike statistics.

This file is collected last on purpose, and it passes alone in a fresh
process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

import snn_inputs as si

pytestmark = pytest.mark.gpu


def per_neuron_stats(steps, ids, n):
    """Spike count, ISI sum and ISI sum of squares (in steps) per neuron."""
    cnt = np.zeros(n, np.uint32)
    s1 = np.zeros(n, np.uint64)
    s2 = np.zeros(n, np.uint64)
    order = np.lexsort((steps, ids))
    st, i = steps[order].astype(np.int64), ids[order]
    np.add.at(cnt, i, 1)
    same = i[1:] == i[:-1]
    isi = (st[1:] - st[:-1])[same]
    np.add.at(s1, i[1:][same], isi.astype(np.uint64))
    np.add.at(s2, i[1:][same], (isi * isi).astype(np.uint64))
    return cnt, s1, s2


def test_static_scratch_rate_cv_matches_snn_stats(gpu):
    import torch

    prob = si.brunel_12k5(seed=2, n_steps=2000)
    net = gpu.Network(prob, stats=True, log_capacity=1 << 22)
    net.step(200)
    net.stats_clear()
    net.step(1800)
    rate_ref, cv_ref = net.stats(0)
    steps, ids = net.spikes(200, 2000)
    net.close()
    assert rate_ref > 1.0 and cv_ref > 0.0

    cnt, s1, s2 = per_neuron_stats(steps, ids, prob.n)
    dev = torch.device("cuda:0")
    d_cnt = torch.from_numpy(cnt.view(np.int32)).to(dev)
    d_s1 = torch.from_numpy(s1.view(np.int64)).to(dev)
    d_s2 = torch.from_numpy(s2.view(np.int64)).to(dev)
    stream = torch.cuda.current_stream(dev)
    lib = gpu.load()
    results = []
    for _ in range(2):  # the second call sees the first call's leftovers in the shared array
        r, c = ctypes.c_double(-1.0), ctypes.c_double(-1.0)
        st = lib.snn_rate_cv_static(d_cnt.data_ptr(), d_s1.data_ptr(), d_s2.data_ptr(), prob.n, 1800,
                                    prob.instances[0].dt, stream.cuda_stream, ctypes.byref(r), ctypes.byref(c))
        assert st == 0
        results.append((r.value, c.value))
        assert abs(r.value - rate_ref) <= 1e-9 * rate_ref
        assert abs(c.value - cv_ref) <= 1e-9
    assert results[0] == results[1]  # fixed summation order: identical results

    # sizes beyond the static array are refused before any device work
    r, c = ctypes.c_double(), ctypes.c_double()
    assert lib.snn_rate_cv_static(d_cnt.data_ptr(), d_s1.data_ptr(), d_s2.data_ptr(), 16_777_217, 1800, 0.1,
                                  stream.cuda_stream, ctypes.byref(r), ctypes.byref(c)) == -1
