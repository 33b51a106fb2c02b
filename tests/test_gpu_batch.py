"""Batches: many programs iterated in lockstep by shared launches, each with its own
Algorithm 1 state.  A program solved in a batch follows exactly the iterations it
follows alone with the same grid (same kernels, same block split, same reductions),
and its solution passes the oracle's KKT evaluator."""
import numpy as np
import pytest

import oracle
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu

G = 8  # blocks per launch shared by the programs of a batch


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _kkt_ok(p, x, y, tol):
    k = oracle.kkt(p, x, y)
    return max(k["err_p"], k["err_d"], k["err_gap"]) <= tol * 1.01


def _solve_batch(probs, tol, max_iter=200_000):
    solvers = [P.Solver(p, batch_blocks=G) for p in probs]
    b = P.Batch(solvers)
    st, nconv = b.solve(tol, max_iter)
    out = [(s.solution(), s.info()) for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    return st, nconv, out


def test_lasso_batch_equals_single_solves_and_passes_the_oracle():
    probs = I.lasso_batch(3, 10, 20, 120)
    st, nconv, res = _solve_batch(probs, 1e-6)
    assert st == P.OK and nconv == len(probs)
    for p, ((x, y), info) in zip(probs, res):
        assert _kkt_ok(p, x, y, 1e-6)
        alone = P.Solver(p, batch_blocks=G)
        st1, info1 = alone.solve(1e-6, 200_000)
        x1, y1 = alone.solution()
        alone.close()
        assert st1 == P.OK
        assert info1["attempts"] == info["attempts"] and info1["restarts"] == info["restarts"]
        np.testing.assert_array_equal(x, x1)
        np.testing.assert_array_equal(y, y1)


def test_batch_of_different_cone_mixes():
    probs = [I.small_socp(0), I.edge_cases(5), I.scaled_mixed_cone(1, 0.01), I.lasso_socp(9, 80)]
    st, nconv, res = _solve_batch(probs, 1e-6, 400_000)
    assert st == P.OK and nconv == len(probs)
    for p, ((x, y), info) in zip(probs, res):
        assert _kkt_ok(p, x, y, 1e-6), p["name"]
        if "obj_star" in p:
            assert abs(oracle.kkt(p, x, y)["pobj"] - p["obj_star"]) <= 1e-5 * (1 + abs(p["obj_star"]))


def test_batch_iterations_follow_the_oracle():
    """The first evaluations of a batched program match the FP64 oracle as a single
    program's do (iteration parity through the batched launches)."""
    p = I.lasso_socp(4, 40)
    s = P.Solver(p, batch_blocks=G, check_period=16)
    other = P.Solver(I.lasso_socp(5, 70), batch_blocks=G, check_period=16)
    b = P.Batch([s, other])
    b.solve(0.0, 16)
    o = oracle.Solver(p, check_period=16)
    o.run(16)
    gx, gy, _, _ = s.iterate()
    ox, oy, _, _ = o.iterate()
    sc = max(1.0, np.abs(ox).max(), np.abs(oy).max())
    assert max(np.abs(gx - ox).max(), np.abs(gy - oy).max()) <= 1e-12 * sc
    b.close()
    s.close()
    other.close()


def test_batch_rejects_mismatched_programs():
    a = P.Solver(I.lasso_socp(1, 30), batch_blocks=G)
    c = P.Solver(I.lasso_socp(2, 30), batch_blocks=G + 1)
    with pytest.raises(P.PdcsError):
        P.Batch([a, c])
    d = P.Solver(I.lasso_socp(3, 30))  # no shared grid
    with pytest.raises(P.PdcsError):
        P.Batch([a, d])
    for s in (a, c, d):
        s.close()
