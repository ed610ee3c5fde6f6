"""Pins of the oracle's tutorial model (Section III-B, Listing 1).

The model: the first population of an instance starts active; a neuron
fires at the step after it received input and not again until it receives
more, so activity hops from one population to its out-neighbours every d
steps.  Pinned by hand-worked rasters, breadth-first search over the graph,
and the binary32 oracle's LIF relay form of the same graph.
"""
import numpy as np
import pytest

import oracle
import snn_inputs as si
from test_oracle_pins import _problem, _relay_problem, _state


def _raster(out):
    r = {}
    for s, i in zip(out["steps"].tolist(), out["ids"].tolist()):
        r.setdefault(s, []).append(i)
    return r


def _tiny(d, n_steps, edges, w, n=4, n_first=1):
    inst = si.brunel_instance(n, k=0)
    inst.n_exc = n_first
    prob = _problem(si.BRUNEL, inst, n_steps=n_steps, delay=d, edges=edges, w=w)
    prob.model = 2
    return prob


@pytest.mark.parametrize("d,expect", [
    (1, {0: [0], 1: [1], 2: [2, 3], 3: [0], 4: [1], 5: [2, 3]}),
    (2, {0: [0], 2: [1], 4: [2, 3], 6: [0]}),
])
def test_hand_worked_rasters(d, expect):
    """0 -> 1, 1 -> 2, 1 -> 3, 2 -> 0; neuron 0 starts active."""
    prob = _tiny(d, 6 if d == 1 else 7, [(0, 1), (1, 2), (1, 3), (2, 0)], [5, 5, 5, 5])
    out = oracle.relay_raster(prob)
    assert _raster(out) == expect
    # events: rows delivered inside the run (a spike of step t at t + d - 1)
    T = prob.n_steps
    rows = {0: 1, 1: 2, 2: 1, 3: 0}
    assert out["events"] == sum(rows[i] for t, ids in expect.items() for i in ids if t + d - 1 <= T - 1)


def test_inputs_that_cancel_do_not_fire():
    """The update sees the summed weights: +7 and -7 in one delivery is no
    input; +7 and -3 is."""
    prob = _tiny(1, 3, [(0, 2), (1, 2), (0, 3), (1, 3)], [7, -7, 7, -3], n_first=2)
    assert _raster(oracle.relay_raster(prob)) == {0: [0, 1], 1: [3]}


@pytest.mark.parametrize("d", [1, 2, 5])
def test_two_populations_match_bfs(d):
    """Listing 1's two populations of 100, randomly connected A -> B and B -> A."""
    prob, edges = _relay_problem(100, 100, 0.05, d, 60, seed=3)
    prob.instances[0].n_exc = 100
    prob.model = 2
    out = oracle.relay_raster(prob)
    succ = {j: set() for j in range(200)}
    for j, i in edges:
        succ[j].add(i)
    frontier, expect, t = set(range(100)), {0: set(range(100))}, 0
    while t + d < 60:
        frontier = set().union(*[succ[j] for j in frontier]) if frontier else set()
        t += d
        expect[t] = frontier
    assert any(len(v) for k, v in expect.items() if k > 20)
    got = _raster(out)
    for t in range(60):
        assert set(got.get(t, [])) == expect.get(t, set()), t


@pytest.mark.parametrize("d", [1, 3])
def test_equals_the_lif_relay_form(d):
    """The binary32 oracle's LIF relay (no leak memory, threshold below one
    weight, no refractory period, population A given input before step 0)
    fires at the same steps and delivers the same events."""
    prob, edges = _relay_problem(100, 100, 0.05, d, 40, seed=1)
    acc0 = np.zeros(200, np.int32)
    acc0[:100] = 6554
    lif = oracle.run(prob, state=_state(200, acc0=acc0, w=[6554] * len(edges)))
    prob.instances[0].n_exc = 100
    prob.model = 2
    rel = oracle.relay_raster(prob)
    assert np.array_equal(lif["steps"], rel["steps"]) and np.array_equal(lif["ids"], rel["ids"])
    assert lif["events"] == rel["events"]
    assert np.array_equal(np.asarray(lif["acc0"], np.int64), rel["acc0"])
