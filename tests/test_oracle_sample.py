"""The CPU baseline's parallel sample: network b of a batched sweep, rebuilt
alone, is the same network as inside the batch (graph and Philox keys), so
the processes of the sample step exactly the sweep's first networks."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import snn_inputs as si  # noqa: E402


def test_network_rebuilt_alone_equals_its_part_of_the_batch():
    kw = dict(n_lo=300, n_hi=2000)
    full = si.batched_sweep(5, base_seed=3, n_steps=0, **kw)
    params = si.batched_sweep_params(5, 3, **kw)
    for b in range(5):
        part = si.sub_problem(full, b)
        alone = si.problem(si.BRUNEL, [params[b]], delay=15, n_steps=0, seed=3, threads=1, inst_index0=b)
        assert np.array_equal(part.row_off, alone.row_off)
        assert np.array_equal(part.tgt, alone.tgt)
        assert np.array_equal(part.w, alone.w)
    # and the oracle steps it as it steps that network inside the batch
    b = 2
    part = si.sub_problem(full, b, n_steps=150)
    alone = si.problem(si.BRUNEL, [params[b]], delay=15, n_steps=150, seed=3, threads=1, inst_index0=b)
    o_part, o_alone = oracle.run(part, inst_key0=b), oracle.run(alone, inst_key0=b)
    assert o_part["events"] == o_alone["events"] > 0
    assert np.array_equal(o_part["ids"], o_alone["ids"])
    whole = oracle.run(si.batched_sweep(5, base_seed=3, n_steps=150, **kw))
    lo, hi = int(full.inst_off[b]), int(full.inst_off[b + 1])
    sel = (whole["ids"] >= lo) & (whole["ids"] < hi)
    assert np.array_equal(whole["ids"][sel] - lo, o_alone["ids"])
    assert np.array_equal(whole["steps"][sel], o_alone["steps"])


def test_window_sample_counts_the_serial_events():
    """oracle_window over the first networks of a 3-network sweep (one
    process each) times steps [t0, t0 + k) of each network as the difference
    of two runs from step 0: its events per process are the serial oracle's
    events of that window, and its value the sum of the per-process rates."""
    import bench
    t0, k_min = 40, 80
    r = bench.oracle_window("batched_sweep_3", 0, t0, k_min, None, timeout_s=600)
    assert r is not None
    value, cores, desc, secs, k, per = r
    n = min(3, len(os.sched_getaffinity(0)))
    assert cores == n and secs > 0 and k == k_min and len(per) == n
    params = si.batched_sweep_params(3, bench.replica_seed(0))
    for b, kb, ev, dt in per:
        assert kb == k_min and dt > 0
        p = si.problem(si.BRUNEL, [params[b]], delay=15, n_steps=t0, seed=bench.replica_seed(0), threads=1,
                       inst_index0=b)
        e_a = oracle.run(p, inst_key0=b)["events"]
        p.n_steps = t0 + k_min
        e_b = oracle.run(p, inst_key0=b)["events"]
        assert ev == e_b - e_a > 0
    assert abs(value - sum(ev / dt for _, _, ev, dt in per)) <= 1e-9 * value
    assert f"networks 0-{n - 1}" in desc and f"steps [{t0}, {t0 + k_min})" in desc


def test_reference_arm_line():
    """`bench.py --impl reference` prints one JSON line with the reference
    arm's keys: the oracle's rate on the parallel sample, its cores and
    sample, and an end-to-end entry that moves no bytes."""
    import json
    import subprocess
    env = dict(os.environ)
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        env.pop(k, None)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "batched_sweep_4", "--steps", "20", "--warmup", "3", "--ref-seconds", "2"],
                       capture_output=True, text=True,
                       env=env, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [x for x in r.stdout.splitlines() if x.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "synaptic events/s" and d["higher_is_better"] is True
    assert d["value"] > 0 and d["steps"] == 20 and d["warmup"] == 3
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["value"] == d["value"]
    assert cb["cores"] == min(4, len(os.sched_getaffinity(0)))
    # the window starts after the settle and warm-up steps and lasts at least 100 steps
    assert d["config"]["window"][0] == 200 + 3 and d["config"]["window"][1] - d["config"]["window"][0] >= 100
    assert "timed as the difference of two runs from step 0" in cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
