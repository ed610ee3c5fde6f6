"""Parity of the GPU adjacency construction (snn_expand_jobs, Fig. 2) with
the oracle: the same jobs and seed give the same integers, bit for bit."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


def _jobs(rng, count, o0=0, width_hi=5000, a_hi=100000):
    jobs = np.zeros(count, dtype=oracle.JOB_DTYPE)
    o = o0
    for j in range(count):
        a = int(rng.integers(0, a_hi))
        width = int(rng.integers(1, width_hi))
        n = int(rng.integers(0, width + 1))
        jobs[j] = (n, a, a + width, 0, o)
        o += n
    return jobs, o


def _gpu(gpu, jobs, seed, out_len):
    import torch
    out = torch.full((max(out_len, 1),), -1, dtype=torch.int32, device="cuda")
    gpu.expand_jobs(jobs.view(gpu.JOB_DTYPE) if jobs.dtype != gpu.JOB_DTYPE else jobs, seed, out_len, out=out)
    torch.cuda.synchronize()
    return out[:out_len].cpu().numpy().view(np.uint32)


@pytest.mark.parametrize("seed", [1, 12345])
def test_random_jobs_match_the_oracle(gpu, seed):
    rng = np.random.default_rng(seed)
    jobs, total = _jobs(rng, 2000, o0=5)
    o = oracle.expand_jobs(jobs, seed=seed, out_len=total + 3)
    g = _gpu(gpu, jobs, seed, total + 3)
    assert np.array_equal(g, o)


def test_long_jobs_and_edges(gpu):
    """Jobs longer than one pass of the warp (256 spacings) and several of
    them, full ranges, an empty job, the largest scale (2^24), and the sizes
    around the lanes' 32 spacings and the one-pass limit (1,024 spacings)."""
    specs = [(0, 0, 10), (1, 0, 1), (50, 100, 150), (255, 0, 300), (256, 7, 10000), (257, 0, 1 << 20),
             (100000, 5, 5 + 100000 + (1 << 24)), (70000, 0, 70000), (3, 0, 3), (1000, 123, 2000),
             (31, 0, 40), (32, 9, 100), (33, 0, 33), (1022, 0, 5000), (1023, 17, 1 << 24), (1024, 0, 1024),
             (1025, 3, 9000)]
    jobs = np.zeros(len(specs), dtype=oracle.JOB_DTYPE)
    o = 0
    for i, (n, a, b) in enumerate(specs):
        jobs[i] = (n, a, b, 0, o)
        o += n
    ref = oracle.expand_jobs(jobs, seed=7, out_len=o)
    g = _gpu(gpu, jobs, 7, o)
    assert np.array_equal(g, ref)
    full = 1 + 50 + 255 + 256 + 257 + 100000  # offset of the 70,000-of-70,000 job
    one = sum(n for n, _, _ in specs[:15])  # offset of the 1,024-of-1,024 job
    assert g[one:one + 1024].tolist() == list(range(1024))
    assert g[full:full + 70000].tolist() == list(range(70000))


def test_many_short_jobs(gpu):
    """One job per neuron of a 20,000-neuron network, out-degree ~100 from
    its own instance range: the shape of a graph build."""
    rng = np.random.default_rng(3)
    n_jobs = 20000
    deg = rng.binomial(2000, 0.05, n_jobs).astype(np.uint32)
    jobs = np.zeros(n_jobs, dtype=oracle.JOB_DTYPE)
    jobs["n"], jobs["a"], jobs["b"] = deg, 0, 2000
    jobs["o"] = np.concatenate([[0], np.cumsum(deg.astype(np.uint64))[:-1]])
    total = int(deg.sum())
    ref = oracle.expand_jobs(jobs, seed=99, out_len=total)
    g = _gpu(gpu, jobs, 99, total)
    assert np.array_equal(g, ref)


def test_invalid_jobs_are_rejected(gpu):
    """A job that does not fit is reported and writes nothing; the valid jobs
    of the same call are written."""
    jobs = np.zeros(3, dtype=oracle.JOB_DTYPE)
    jobs[0] = (5, 0, 10, 0, 0)
    jobs[1] = (20, 0, 10, 0, 5)  # more values than the range holds
    jobs[2] = (5, 0, 10, 0, 28)  # past the end of the output
    import torch
    out = torch.full((30,), -1, dtype=torch.int32, device="cuda")
    with pytest.raises(gpu.SnnError):
        gpu.expand_jobs(jobs, 1, 30, out=out)
    g = out.cpu().numpy().view(np.uint32)
    ref = oracle.expand_jobs(jobs[:1], seed=1, out_len=5)
    assert np.array_equal(g[:5], ref)
    assert np.all(g[5:] == 0xffffffff)
