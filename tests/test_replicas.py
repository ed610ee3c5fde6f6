"""The multi-GPU path of bench.py is replicas: each rank simulates its own
networks (distinct graph seeds) and only the timing is combined -- the
slowest rank's time and the sum of the events.  Tested here with two gloo
ranks on the CPU (no GPU, no NCCL)."""
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import bench
    import snn_inputs as si

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        events = [1000.0, 3000.0][rank]
        seconds = [0.5, 0.8][rank]
        out[rank] = {
            "max": bench.reduce_over_ranks(seconds, "max", dist, "cpu"),
            "sum": bench.reduce_over_ranks(events, "sum", dist, "cpu"),
            "value": bench.replica_value(events, seconds, dist, "cpu"),
            "sizes": [inst.n for inst in si.batched_sweep_params(4, base_seed=bench.replica_seed(rank))],
        }
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_replicas_combine_time_and_events():
    port = 29000 + os.getpid() % 1000
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        r0, r1 = out[0], out[1]
    assert r0["max"] == r1["max"] == 0.8
    assert r0["sum"] == r1["sum"] == 4000.0
    assert r0["value"] == r1["value"] == 4000.0 / 0.8
    assert r0["sizes"] != r1["sizes"]  # each replica has its own networks


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.reduce_over_ranks(2.5, "max", None, "cpu") == 2.5
    assert bench.replica_value(10.0, 2.0, None, "cpu") == 5.0


def test_reference_arm_runs_on_rank_zero_only():
    """Under torchrun the reference arm (the oracle) runs on rank 0 alone; the
    other ranks exit at once, printing nothing."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
