"""The binary32 lattice oracle against the binary64 float-weight variant.

Both variants see the same graph and the same Poisson draws; they differ in
state precision and in weight quantisation.  The runs are chaotic, so their
rasters part ways; what must agree is the statistics that characterise the
paper's models (population rate, ISI irregularity): pooled over seeds, the rate
within 2 % and the mean ISI CV within 5 %.
"""
import numpy as np
import pytest

import oracle
import snn_inputs as si


def rate_and_cv(steps, ids, n, T, dt_ms, skip=0.1):
    """Population rate (Hz) and mean ISI CV over neurons with >= 3 spikes,
    after discarding the first `skip` fraction of the steps."""
    t0 = int(T * skip)
    m = steps >= t0
    rate = m.sum() / n / ((T - t0) * dt_ms * 1e-3)
    s, i = steps[m], ids[m]
    order = np.lexsort((s, i))
    s, i = s[order].astype(np.float64), i[order]
    starts = np.flatnonzero(np.r_[True, i[1:] != i[:-1]])
    ends = np.r_[starts[1:], len(i)]
    cvs = [np.diff(s[a:b]).std() / np.diff(s[a:b]).mean() for a, b in zip(starts, ends) if b - a >= 3]
    return rate, float(np.mean(cvs))


@pytest.mark.parametrize("name,make,T", [
    ("vogels_4k", lambda sd: si.vogels_4k(seed=sd, n_steps=10000), 10000),
    ("brunel_12k5", lambda sd: si.brunel_12k5(seed=sd, n_steps=3000), 3000),
])
def test_f32_lattice_statistics_match_f64(name, make, T):
    r32, r64, c32, c64 = [], [], [], []
    for seed in (1, 2, 3):
        p = make(seed)
        a = oracle.run(p)
        b = oracle.run_f64(p)
        ra, ca = rate_and_cv(a["steps"], a["ids"], p.n, T, 0.1)
        rb, cb = rate_and_cv(b["steps"], b["ids"], p.n, T, 0.1)
        r32.append(ra); r64.append(rb); c32.append(ca); c64.append(cb)
        assert rb > 1.0  # the networks are active
    assert abs(np.mean(r32) / np.mean(r64) - 1) < 0.02
    assert abs(np.mean(c32) / np.mean(c64) - 1) < 0.05
