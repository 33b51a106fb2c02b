"""FP32-iterate mode: SpMV, updates and cone projections on FP32 iterates, with the
restart / termination checks (candidates, their products, KKT residuals) and the final
phase in FP64.  Results are checked by the FP64 oracle's KKT evaluator."""
import numpy as np
import pytest

import oracle
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _kkt_max(p, x, y):
    k = oracle.kkt(p, x, y)
    return max(k["err_p"], k["err_d"], k["err_gap"]), k


@pytest.mark.parametrize("prob_name", ["small_socp", "mixed_small", "edge_cases"])
def test_fp32_mode_with_fp64_polish_reaches_1e6(prob_name):
    p = {"small_socp": lambda: I.small_socp(0), "mixed_small": lambda: I.scaled_mixed_cone(1, 0.01),
         "edge_cases": lambda: I.edge_cases(5)}[prob_name]()
    g = P.Solver(p, precision=P.PRECISION_FP32)
    st, info = g.solve(1e-6, 400_000)
    assert st == P.OK, info
    assert info["fp64_phase"] == 1  # 1e-6 lies below the FP32 phase's switch point
    x, y = g.solution()
    err, k = _kkt_max(p, x, y)
    assert err <= 1.01e-6
    assert abs(k["pobj"] - p["obj_star"]) <= 1e-5 * (1 + abs(p["obj_star"]))
    g.close()


def test_fp32_mode_alone_at_a_loose_tolerance():
    p = I.scaled_mixed_cone(1, 0.01)
    g = P.Solver(p, precision=P.PRECISION_FP32, fp32_switch_tol=1e-5)
    st, info = g.solve(1e-3, 200_000)
    assert st == P.OK, info
    assert info["fp64_phase"] == 0  # never left FP32
    x, y = g.solution()
    err, _ = _kkt_max(p, x, y)
    assert err <= 1.01e-3  # the FP64 check's verdict agrees with the oracle's evaluator
    g.close()


def test_fp32_iterates_track_the_fp64_oracle():
    """The first evaluations in FP32 stay within FP32 rounding (amplified by the
    adaptive step) of the FP64 oracle's iterates."""
    p = I.small_socp(0)
    g = P.Solver(p, precision=P.PRECISION_FP32, check_period=16)
    o = oracle.Solver(p, check_period=16)
    for n in [1, 4, 8]:
        g.run(n - g.info()["attempts"])
        o.run(n - o.scalars()["attempts"])
        gx, gy, _, _ = g.iterate()
        ox, oy, _, _ = o.iterate()
        sc = max(1.0, np.abs(ox).max(), np.abs(oy).max())
        err = max(np.abs(gx - ox).max(), np.abs(gy - oy).max()) / sc
        assert err <= 1e-4, (n, err)
    g.close()


def test_fp32_mode_warm_start_at_optimum():
    p = I.small_socp(0)
    g = P.Solver(p, precision=P.PRECISION_FP32)
    g.warm_start(p["x_star"], p["y_star"])
    st, info = g.solve(1e-6, 20_000)
    assert st == P.OK, info
    x, y = g.solution()
    err, _ = _kkt_max(p, x, y)
    assert err <= 1.01e-6
    g.close()
