"""Pins of the oracle's adjacency construction (Section III-A-2, Fig. 2):
the worked example of the figure, the mathematics the method rests on (the
normalised running sums of exponential spacings are uniform order
statistics) and the invariants of its output."""
import math
import os

import numpy as np
import pytest
from scipy import stats

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fig2_job_expansion.txt")


def _fig2():
    rows = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, *vals = line.split()
            rows[key] = [None if v == "-" else float(v) for v in vals]
    return rows


def test_fig2_negative_logarithm():
    """(a) -> (b): each printed spacing is -ln of its printed draw, to the
    printed two decimals."""
    f = _fig2()
    for u, b in zip(f["a"], f["b"]):
        assert abs(oracle.neg_ln(u) - b) <= 0.005 + 1e-6, (u, b)


def test_fig2_running_sum():
    """(a) -> (c): the running sum of the spacings starts at 0 (the first
    sentinel) and its last entry (the second sentinel) is the sum of all but
    the last spacing."""
    f = _fig2()
    q, c, _ = oracle.job_from_uniforms(f["a"][:7], 0, 100)
    got = c.astype(np.float64) / 2**22
    assert got[0] == 0.0
    assert np.all(np.abs(got - np.array(f["c"])) <= 0.005 + 1e-6), got


def test_fig2_scale_round_offsets():
    """(d) -> (g): with draws whose normalised running sums are the printed
    (d), the oracle scales by b - a - n = 94, rounds (e), adds 0..5 (f) and
    returns the printed (g)."""
    f = _fig2()
    d = np.array(f["d"])
    spacing = np.diff(d) * 4.0  # any total: only the ratios matter
    u = np.exp(-spacing).astype(np.float32)
    _, c, out = oracle.job_from_uniforms(u, 0, 100)
    ratio = c.astype(np.float64) / float(c[-1])
    assert np.allclose(ratio, d, atol=1e-6)
    assert [int(round(x * 94)) for x in d] == [int(v) for v in f["e"]]
    assert out.tolist() == [int(v) for v in f["g"][1:-1]]


def test_negative_logarithm_accuracy():
    """The oracle's own binary32 logarithm against the library's binary64
    one: within a few units in the last place over (0, 1]."""
    rng = np.random.default_rng(3)
    us = np.concatenate([(rng.integers(0, 2**24, 20000) + 1) / 2.0**24,
                         [2.0**-24, 0.5, 0.75, 1.0 - 2.0**-24, 1.0]]).astype(np.float32)
    for u in us:
        ref = -math.log(float(u))
        got = oracle.neg_ln(float(u))
        assert abs(got - ref) <= 4e-7 * max(1.0, ref), (u, got, ref)
    assert oracle.neg_ln(1.0) == 0.0


def _random_jobs(rng, count, o0=0):
    jobs = np.zeros(count, dtype=oracle.JOB_DTYPE)
    o = o0
    for j in range(count):
        a = int(rng.integers(0, 1000))
        width = int(rng.integers(1, 5000))
        n = int(rng.integers(0, width + 1))
        jobs[j] = (n, a, a + width, 0, o)
        o += n
    return jobs, o


def test_job_invariants():
    """Each job writes exactly its n slots with strictly increasing values in
    [a, b); slots of no job stay untouched."""
    rng = np.random.default_rng(5)
    jobs, total = _random_jobs(rng, 300, o0=7)
    out = oracle.expand_jobs(jobs, seed=11, out_len=total + 9)
    assert np.all(out[:7] == 0xffffffff) and np.all(out[total:] == 0xffffffff)
    for n, a, b, _, o in jobs:
        v = out[o:o + n].astype(np.int64)
        assert v.size == n
        if n:
            assert v[0] >= a and v[-1] < b
            assert np.all(np.diff(v) > 0)


def test_job_full_and_empty_ranges():
    """n = b - a leaves no freedom (a, a+1, ..., b-1); n = 0 writes nothing."""
    jobs = np.zeros(3, dtype=oracle.JOB_DTYPE)
    jobs[0] = (50, 100, 150, 0, 0)
    jobs[1] = (0, 7, 9, 0, 50)
    jobs[2] = (1, 3, 4, 0, 50)
    out = oracle.expand_jobs(jobs, seed=2, out_len=51)
    assert out[:50].tolist() == list(range(100, 150))
    assert out[50] == 3


def _binned_beta(k: int, n: int, M: int) -> np.ndarray:
    """P(round(M x) = j), j = 0..M, for x the k-th smallest of n uniforms
    (x ~ Beta(k, n + 1 - k)): the law of the k-th value minus (a + k - 1)."""
    edges = np.clip((np.arange(M + 2) - 0.5) / M, 0.0, 1.0)
    return np.diff(stats.beta.cdf(edges, k, n + 1 - k))


def _chisquare(counts, probs):
    exp = probs * counts.sum()
    keep = exp >= 5
    obs = np.append(counts[keep], counts[~keep].sum())
    e = np.append(exp[keep], exp[~keep].sum())
    if e[-1] == 0:
        obs, e = obs[:-1], e[:-1]
    return stats.chisquare(obs, e).pvalue


def test_job_single_value_law():
    """n = 1 from [0, 10): the normalised spacing is uniform on [0, 1], so
    round(9 x) puts weight 1/9 on 1..8 and 1/18 on each end (the printed
    method scales and rounds)."""
    jobs = np.zeros(20000, dtype=oracle.JOB_DTYPE)
    jobs["n"], jobs["a"], jobs["b"] = 1, 0, 10
    jobs["o"] = np.arange(20000)
    out = oracle.expand_jobs(jobs, seed=4, out_len=20000)
    counts = np.bincount(out, minlength=10)
    assert _chisquare(counts, _binned_beta(1, 1, 9)) > 1e-4, counts


def test_job_order_statistics():
    """n = 5 from [0, 25): the k-th value minus (k - 1) is round(20 x_k) with
    x_k the k-th order statistic of 5 uniforms -- the fact the method rests
    on (running sums of exponential spacings, normalised, are uniform order
    statistics)."""
    n, M, J = 5, 20, 20000
    jobs = np.zeros(J, dtype=oracle.JOB_DTYPE)
    jobs["n"], jobs["a"], jobs["b"] = n, 0, M + n
    jobs["o"] = np.arange(J) * n
    out = oracle.expand_jobs(jobs, seed=8, out_len=J * n).reshape(J, n).astype(np.int64)
    for k in range(1, n + 1):
        r = out[:, k - 1] - (k - 1)
        counts = np.bincount(r, minlength=M + 1)
        assert _chisquare(counts, _binned_beta(k, n, M)) > 1e-4, (k, counts)


def test_job_rejects_bad_jobs():
    bad = np.zeros(1, dtype=oracle.JOB_DTYPE)
    bad[0] = (11, 0, 10, 0, 0)  # more values than the range holds
    with pytest.raises(oracle.OracleError):
        oracle.expand_jobs(bad, seed=1, out_len=20)
    bad[0] = (1, 0, 10, 0, 20)  # outside the output
    with pytest.raises(oracle.OracleError):
        oracle.expand_jobs(bad, seed=1, out_len=20)


def test_a_job_alone_equals_its_part_of_the_list():
    """expand_job(job, j, seed) draws job j's uniforms by its index alone: the
    same values the whole list writes at its offset (what a sampled check of
    a large job list relies on)."""
    rng = np.random.default_rng(11)
    jobs = np.zeros(40, dtype=oracle.JOB_DTYPE)
    o = 0
    for j in range(40):
        a = int(rng.integers(0, 1000))
        w = int(rng.integers(1, 3000))
        n = int(rng.integers(0, w + 1))
        jobs[j] = (n, a, a + w, 0, o)
        o += n
    whole = oracle.expand_jobs(jobs, seed=9, out_len=o)
    for j in range(40):
        lo, n = int(jobs[j]["o"]), int(jobs[j]["n"])
        assert np.array_equal(oracle.expand_job(jobs[j], j, 9), whole[lo:lo + n]), j
