"""The Lasso (dense batched form and the paper's App. B.2 workload), Fisher market (App. B.1)
and portfolio generators, pinned outside the solver: the oracle's optimum of each conic
program equals the optimum an independent method finds for the original problem (coordinate
descent for the Lasso, SLSQP for the Fisher market and the portfolio)."""
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


def test_paper_lasso_program_matches_coordinate_descent():
    """The paper's Lasso workload (App. B.2: sparse U[0, 1] design, half-zero ground truth,
    lam = ||A'b||_inf, one SOC of dimension m + 2), at a small size and a higher density."""
    sk = pytest.importorskip("sklearn.linear_model")
    q = I.lasso_paper(11, m=40, n=400, density=0.05)
    A, b, lam = q["lasso"]["A"].toarray(), q["lasso"]["b"], q["lasso"]["lam"]
    m, n = A.shape
    assert q["cone_dims"][-1] == m + 2 and lam == pytest.approx(np.abs(A.T @ b).max())
    fit = sk.Lasso(alpha=lam / (2 * m), fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(A, b)
    w = fit.coef_
    f_cd = float(np.sum((A @ w - b) ** 2) + lam * np.abs(w).sum())
    f_or, x = _oracle_optimum(q)
    assert abs(f_or - f_cd) <= 1e-6 * max(1.0, abs(f_cd)), (f_or, f_cd)
    i1 = 2 + m
    np.testing.assert_allclose(x[i1:i1 + n] - x[i1 + n:i1 + 2 * n], w, atol=1e-4)


def test_fisher_market_program_matches_slsqp_and_clears_the_budgets():
    """The paper's Fisher market workload (App. B.1) at a small size: the oracle's optimum
    equals the Eisenberg-Gale optimum that SLSQP finds directly, and the equilibrium prices
    (the duals of the clearing rows) spend exactly the buyers' budgets: sum_j p_j b_j = sum_i w_i."""
    q = I.fisher_market(3, buyers=6, goods=10, density=0.5)
    U, w, bs = q["fisher"]["U"].toarray(), q["fisher"]["w"], q["fisher"]["b"]
    mb, ng = U.shape
    rows, cols = np.nonzero(U)  # the program's X variables, row-major as the generator orders them
    u = U[rows, cols]

    def f(xv):
        util = np.bincount(rows, weights=u * xv, minlength=mb)
        return -float(w @ np.log(np.maximum(util, 1e-300)))

    def g(xv):
        util = np.bincount(rows, weights=u * xv, minlength=mb)
        return -(w[rows] * u / np.maximum(util[rows], 1e-300))

    cons = [{"type": "eq", "fun": lambda xv: np.bincount(cols, weights=xv, minlength=ng) - bs,
             "jac": lambda xv: (np.arange(ng)[:, None] == cols[None, :]).astype(float)}]
    x0 = bs[cols] / np.bincount(cols, minlength=ng)[cols]
    r = minimize(f, x0, jac=g, method="SLSQP", bounds=[(0.0, None)] * rows.size, constraints=cons,
                 options={"ftol": 1e-15, "maxiter": 2000})
    assert r.success, r.message
    f_or, x = _oracle_optimum(q, tol=1e-9)
    assert abs(f_or - r.fun) <= 1e-6 * max(1.0, abs(r.fun)), (f_or, r.fun)
    s = oracle.Solver(q)
    assert s.run(2_000_000, 1e-9) == oracle.CONVERGED
    _, y = s.solution()
    assert abs(abs(float(y[:ng] @ bs)) - w.sum()) <= 1e-6 * w.sum()


def test_paper_lasso_with_a_primal_cone_matches_coordinate_descent():
    """The same Lasso with the cone on the variables (the appendix's own form: (w, r, y) in
    K_rsoc as a primal cone block, only the zero rows left): the same optimum."""
    sk = pytest.importorskip("sklearn.linear_model")
    q = I.lasso_paper_kp(11, m=40, n=400, density=0.05)
    A, b, lam = q["lasso"]["A"].toarray(), q["lasso"]["b"], q["lasso"]["lam"]
    m, n = A.shape
    assert q["m"] == m + 1 and q["pcone_dims"][0] == m + 2
    fit = sk.Lasso(alpha=lam / (2 * m), fit_intercept=False, tol=1e-14, max_iter=1_000_000).fit(A, b)
    w = fit.coef_
    f_cd = float(np.sum((A @ w - b) ** 2) + lam * np.abs(w).sum())
    s = oracle.Solver(q, beta=0.5)
    assert s.run(2_000_000, 1e-9) == oracle.CONVERGED
    x, y = s.solution()
    k = oracle.kkt(q, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1e-9
    assert abs(k["pobj"] - f_cd) <= 1e-6 * max(1.0, abs(f_cd)), (k["pobj"], f_cd)
    i1 = 2 + m
    np.testing.assert_allclose(x[i1:i1 + n] - x[i1 + n:i1 + 2 * n], w, atol=1e-4)
