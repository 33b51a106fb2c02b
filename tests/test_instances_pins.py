"""The Lasso (App. C form) and portfolio generators, pinned outside the solver: the
oracle's optimum of each conic program equals the optimum an independent method finds
for the original problem (coordinate descent for the Lasso, SLSQP for the portfolio)."""
import numpy as np
import pytest
from scipy.optimize import minimize

import oracle
from paper_2505_00311_gb300 import instances as I


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _oracle_optimum(q, tol=1e-9):
    s = oracle.Solver(q)
    assert s.run(2_000_000, tol) == oracle.CONVERGED
    x, y = s.solution()
    k = oracle.kkt(q, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= tol
    return k["pobj"], x


@pytest.mark.parametrize("seed,n", [(3, 24), (4, 40)])
def test_lasso_program_matches_coordinate_descent(seed, n):
    sk = pytest.importorskip("sklearn.linear_model")
    q = I.lasso_socp(seed, n)
    A, b, lam = q["lasso"]["A"], q["lasso"]["b"], q["lasso"]["lam"]
    m = A.shape[0]
    # ||A x - b||^2 + lam ||x||_1 = 2m [ ||b - A x||^2 / (2m) + (lam / 2m) ||x||_1 ]
    fit = sk.Lasso(alpha=lam / (2 * m), fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(A, b)
    w = fit.coef_
    f_cd = float(np.sum((A @ w - b) ** 2) + lam * np.abs(w).sum())
    f_or, x = _oracle_optimum(q)
    assert abs(f_or - f_cd) <= 1e-6 * max(1.0, abs(f_cd)), (f_or, f_cd)
    i1 = 2 + m
    np.testing.assert_allclose(x[i1:i1 + n] - x[i1 + n:i1 + 2 * n], w, atol=1e-4)


def test_portfolio_program_matches_slsqp():
    fam = I.portfolio_family(seed=1, n_assets=40, k=4)
    mu = I.portfolio_mu(fam, 0)
    q = I.portfolio_socp(fam, mu)
    F, gamma, cap = fam["F"], fam["gamma"], fam["cap"]
    na = F.shape[0]
    cons = [{"type": "eq", "fun": lambda x: x.sum() - 1.0, "jac": lambda x: np.ones(na)},
            {"type": "ineq", "fun": lambda x: gamma ** 2 - np.sum((F.T @ x) ** 2),
             "jac": lambda x: -2.0 * F @ (F.T @ x)}]
    x0 = np.full(na, 1.0 / na)
    r = minimize(lambda x: -mu @ x, x0, jac=lambda x: -mu, method="SLSQP", bounds=[(0.0, cap)] * na,
                 constraints=cons, options={"ftol": 1e-14, "maxiter": 1000})
    assert r.success, r.message
    f_or, x = _oracle_optimum(q, tol=1e-8)
    assert abs(f_or - r.fun) <= 1e-6 * max(1.0, abs(r.fun)), (f_or, r.fun)
    np.testing.assert_allclose(x[:na], r.x, atol=2e-4)
