"""The counting-scalar build of the oracle (oracle/flop_count.cpp): the
oracle's own C source compiled with a scalar that counts every FP64
operation.  It must compute the oracle's right-hand side to the bit (it is
the oracle), and its counts are the method's FP64 work per zone as the
oracle evaluates it: the algorithmic figure beside the GPU kernels' executed
operation counts."""
import numpy as np

import initial_data as idd
import oracle


def test_counting_build_is_the_oracle_and_counts_per_zone():
    p = idd.single_puncture_patch(16, 8.0)
    u = idd.single_puncture_data(p)
    u[19:22] += 0.1 * np.sin(np.arange(u[0].size).reshape(u[0].shape) * 0.01)[None]  # shift of both signs
    counts, rhs = oracle.flop_counts(p, u)
    assert np.array_equal(rhs, oracle.rhs(p, u, oracle.Params()))
    c = counts
    assert c["points"] == 16 ** 3
    # the parts evaluated one by one add up to the whole right-hand side,
    # up to the additions that join them (a few per field)
    parts = c["sources"]["flops"] + c["advection"]["flops"] + c["dissipation"]["flops"]
    assert c["rhs"]["flops"] <= parts <= c["rhs"]["flops"] + 4 * 25
    # Kreiss-Oliger: 25 fields x 3 directions x (7-point sixth difference on
    # centre differences: 6 differences, 3 sums, 3 weights, 2 adds) + scaling
    assert c["dissipation"]["div"] == 25.0
    # an RK4 stage is the right-hand side plus the update and the constraints
    assert c["rk4_stage_2"]["flops"] > c["rhs"]["flops"]
    assert 6000 < c["rk4_stage_2"]["flops"] < 8000, c
