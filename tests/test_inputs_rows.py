"""The input recipes' one-weight-per-row form (what snn_build_graph_rows
takes): the row weights read back every synapse's weight, the generator's
own record of them agrees with a scan of the weights, and a row with two
weights has no row form."""
import numpy as np

import snn_inputs as si


def test_row_weights_spread_back_to_the_synapse_weights():
    for prob in (si.batched_sweep(n_nets=12, base_seed=3, n_steps=10, n_lo=37, n_hi=6000),
                 si.vogels_4k(seed=2, n_steps=10), si.brunel_stdp_100k(seed=1, n_steps=10, n=3000, k=300)):
        wr = prob.row_weights()
        deg = np.diff(prob.row_off.astype(np.int64))
        assert wr is not None and len(wr) == prob.n
        assert np.array_equal(np.repeat(wr, deg), prob.w)
        assert (wr[deg == 0] == 0).all()
        prob.w = prob.w.copy()  # a new array is scanned again: the same answer
        assert np.array_equal(prob.row_weights(), wr)


def test_sub_problem_and_mixed_rows():
    prob = si.batched_sweep(n_nets=6, base_seed=5, n_steps=10, n_lo=300, n_hi=3000)
    for b in range(6):
        sub = si.sub_problem(prob, b)
        lo, hi = int(prob.inst_off[b]), int(prob.inst_off[b + 1])
        assert np.array_equal(sub.row_weights(), prob.row_weights()[lo:hi])
    w = prob.w.copy()
    e = int(prob.row_off[7])  # first synapse of row 7 (a row with two or more synapses)
    assert prob.row_off[8] - prob.row_off[7] >= 2
    w[e] += 1
    prob.w = w
    assert prob.row_weights() is None
