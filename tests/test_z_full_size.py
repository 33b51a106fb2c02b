"""GPU parity at the benchmark's full size and launch configuration: the 1M-variable
mixed-cone program (n = 1M, m = 500k, ~10M nonzeros, seed 1) with the SpMV autotuner
on and CUDA graphs, as bench.py runs it.  The FP64 oracle manages a few evaluations per
second at this size, so the comparison covers the rescaling, single evaluations from the
oracle's states after 0, 16 and 64 evaluations (per cone role), and the first 16-17
evaluations run side by side, with a restart check inside the window; rounding
differences grow about 10x every 10 evaluations through the adaptive step rule."""
import numpy as np
import pytest

import oracle
from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    oracle.build()


@pytest.fixture(scope="module")
def prob():
    return I.mixed_cone(1)


def rel_inf(a, b):
    return np.max(np.abs(a - b)) / max(1.0, np.max(np.abs(b)))


@pytest.mark.parametrize("check_period", [64, 16])
def test_full_size_scaling_and_first_evaluations(prob, check_period):
    """check_period 64 is the benchmark's configuration (no check inside the window);
    16 puts the first restart check inside it."""
    g = P.Solver(prob, spmv_autotune=1, check_period=check_period)
    o = oracle.Solver(prob, check_period=check_period)
    gdr, gdc = g.scaling()
    odr, odc = o.scaling()
    assert rel_inf(gdr, odr) <= 1e-13 and rel_inf(gdc, odc) <= 1e-13
    done = 0
    for target in [1, 2, 4, 8, 16, 17] if check_period == 16 else [1, 2, 4, 8, 16]:
        g.run(target - done)
        o.run(target - done)
        done = target
        gs, os_ = g.info(), o.scalars()
        assert gs["attempts"] == os_["attempts"]
        assert gs["accepted"] == os_["accepted"] and gs["restarts"] == os_["restarts"], (target, gs, os_)
        err = max(rel_inf(a, b) for a, b in zip(g.iterate(), o.iterate()))
        assert err <= 1e-12, (target, err)
        assert abs(gs["eta"] - os_["eta"]) <= 1e-10 * os_["eta"]
        assert abs(gs["omega"] - os_["omega"]) <= 1e-10 * os_["omega"]
    g.close()


def test_full_size_one_evaluation_from_oracle_states(prob):
    """The oracle's state after 0, 16 and 64 evaluations (a restart check at 64) loaded into
    the library; one evaluation on both; xhat, yhat per cone role (20k exp cones, ~5.9k
    SOCs, 240k scalar rows), the next iterate and step size within 1e-12."""
    from parity_helpers import one_evaluation
    g = P.Solver(prob, spmv_autotune=1, check_period=64)
    o = oracle.Solver(prob, check_period=64)
    done = 0
    for start in [0, 16, 64]:
        o.run(start - done)
        err, acc = one_evaluation(prob, g, o)
        done = start + 1
        assert acc[0] == acc[1], (start, acc, err)
        assert max(err.values()) <= 1e-12, (start, err)
    g.close()
