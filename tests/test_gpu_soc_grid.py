"""The grid-wise projection of large SOC cones (several blocks of one cooperative launch per
cone, Sec. 4's grid-wise strategy) against the FP64 oracle: one PDHG evaluation from the
oracle's states (dual update, candidates and KKT all pass through it), and full solves of the
paper's Lasso workload (App. B.2, one SOC of dimension m + 2) checked by the oracle's KKT
evaluator."""
import numpy as np
import pytest

import oracle
from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu

RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    oracle.build()


@pytest.mark.parametrize("m,n,grid_dim", [(3000, 30_000, 1024), (20_000, 200_000, 0)])
def test_one_evaluation_lasso_grid_wise(m, n, grid_dim):
    """The Lasso SOC (dimension m + 2) split over a team of blocks (forced at 3,002 rows; by
    the default rule at 20,002), one evaluation from the oracle's states after 0, 64 and 200
    evaluations: xhat, yhat per role, the next iterate and step size within 1e-12."""
    from parity_helpers import one_evaluation
    p = I.lasso_paper(5, m=m, n=n, density=2e-4)
    o = oracle.Solver(p, check_period=64)
    g = P.Solver(p, check_period=64, soc_grid_dim=grid_dim)
    assert g.info()["soc_grid_cones"] == 1
    done = 0
    for start in [0, 64, 200]:
        o.run(start - done)
        err, acc = one_evaluation(p, g, o)
        done = start + 1
        assert acc[0] == acc[1] and max(err.values()) <= RTOL, (start, err)
    g.close()


def test_one_evaluation_many_cones_one_block_each():
    """Every SOC / RSOC cone of the mixed-cone program forced onto the grid-wise path: more
    cones than blocks, so each block projects several cones in turn (teams of one block)."""
    from parity_helpers import one_evaluation
    p = I.scaled_mixed_cone(1, 0.05)
    o = oracle.Solver(p, check_period=64)
    g = P.Solver(p, check_period=64, soc_grid_dim=1)
    assert g.info()["soc_grid_cones"] == int(np.sum(np.isin(p["cone_types"], [2, 3])))
    done = 0
    for start in [0, 64]:
        o.run(start - done)
        err, acc = one_evaluation(p, g, o)
        done = start + 1
        assert acc[0] == acc[1] and max(err.values()) <= RTOL, (start, err)
    g.close()


@pytest.mark.parametrize("grid_dim", [1024, -1])
def test_checks_agree_with_the_oracle_evaluator(grid_dim):
    """The KKT errors that a check computes on the device (candidate projections and the
    primal residual's projections through the team kernel, or one warp per cone) equal the
    oracle evaluator's errors of the solution that check returns."""
    p = I.lasso_paper(7, m=3000, n=30_000, density=2e-4)
    g = P.Solver(p, check_period=64, soc_grid_dim=grid_dim)
    assert g.info()["soc_grid_cones"] == (1 if grid_dim > 0 else 0)
    for evals in (64, 640):
        st, info = g.solve(0.0, 64 if evals == 64 else 576)
        x, y = g.solution()
        k = oracle.kkt(p, x, y)
        for q in ("err_p", "err_d", "err_gap"):
            assert abs(info[q] - k[q]) <= 1e-7 * k[q] + 1e-14, (evals, q, info[q], k[q])
    g.close()


def test_lasso_solve_passes_the_oracle_evaluator():
    """A full solve of a 1/10-paper-size Lasso (7,000 x 70,000, 4.9e4 entries of A; the SOC of
    7,002 rows grid-wise) to 1e-5: the returned point meets the tolerance by the oracle's KKT
    evaluator, and its objective matches the Lasso optimum that L-BFGS-B finds on the original
    problem (x = x1 - x2, x1, x2 >= 0)."""
    from scipy.optimize import minimize
    p = I.lasso_paper(0, m=7000, n=70_000, density=1e-4)
    g = P.Solver(p)
    st, info = g.solve(1e-5, 2_000_000)
    assert st == P.OK and info["soc_grid_cones"] == 1
    x, y = g.solution()
    k = oracle.kkt(p, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1e-5, k
    A, b, lam = p["lasso"]["A"].tocsr(), p["lasso"]["b"], p["lasso"]["lam"]
    n = A.shape[1]

    def f(z):
        r = A @ (z[:n] - z[n:]) - b
        gr = 2.0 * (A.T @ r)
        return float(r @ r + lam * z.sum()), np.concatenate([gr + lam, -gr + lam])

    res = minimize(f, np.zeros(2 * n), jac=True, method="L-BFGS-B", bounds=[(0.0, None)] * (2 * n),
                   options={"maxiter": 20000, "ftol": 1e-15, "gtol": 1e-12})
    assert abs(k["pobj"] - res.fun) <= 1e-4 * max(1.0, abs(res.fun)), (k["pobj"], res.fun)
    g.close()


def test_one_evaluation_rotated_cone_across_blocks():
    """A rotated SOC (the dense Lasso's (w, r, y) block of 1,502 rows) split over a team of three
    blocks (soc_grid_dim forces it): the Q transform of the first two rows happens in the first
    block while the others hold the rest of the cone; one evaluation from the oracle's states
    after 0 and 64 evaluations within 1e-12."""
    from parity_helpers import one_evaluation
    p = I.lasso_socp(6, 3000)
    assert p["cone_types"][-1] == 3 and p["cone_dims"][-1] == 1502
    o = oracle.Solver(p, check_period=64)
    g = P.Solver(p, check_period=64, soc_grid_dim=1024)
    assert g.info()["soc_grid_cones"] == 1
    done = 0
    for start in [0, 64]:
        o.run(start - done)
        err, acc = one_evaluation(p, g, o)
        done = start + 1
        assert acc[0] == acc[1] and max(err.values()) <= RTOL, (start, err)
    g.close()
