"""The exponential-cone logistic-regression program (l1-regularised logistic regression
lifted with two exp cones and one nonnegative row per sample, Sec. 5's exp-cone
experiments in synthetic form).  Pinned against the logistic objective itself, outside
the solver: the lifted point of any weight vector lies on the cones' boundary with the
logistic loss as its objective, and the oracle's optimum equals the minimum that a
quasi-Newton method finds for the logistic objective directly."""
import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.special import expit

import oracle
from paper_2505_00311_gb300 import instances as I


def logistic_objective(q, w):
    X, b, lam = q["logistic"]["X"], q["logistic"]["labels"], q["logistic"]["lam"]
    return float(np.logaddexp(0.0, -b * (X @ w)).sum() + lam * np.abs(w).sum())


def logistic_minimum(q):
    """min over w of the logistic objective, by L-BFGS-B on the split w = w+ - w- >= 0."""
    X, b, lam = q["logistic"]["X"], q["logistic"]["labels"], q["logistic"]["lam"]
    p = X.shape[1]

    def f(z):
        mg = -b * (X @ (z[:p] - z[p:]))
        g = X.T @ (-b * expit(mg))
        return np.logaddexp(0.0, mg).sum() + lam * z.sum(), np.concatenate([g + lam, lam - g])

    r = minimize(f, np.zeros(2 * p), jac=True, method="L-BFGS-B", bounds=[(0.0, None)] * (2 * p),
                 options={"ftol": 1e-15, "gtol": 1e-12, "maxiter": 20000})
    return float(r.fun), r.x[:p] - r.x[p:]


def lift(q, w):
    """The program's variables for weights w: t_i the logistic loss of sample i, u, v on
    the boundaries of their exp cones."""
    X, b = q["logistic"]["X"], q["logistic"]["labels"]
    mg = -b * (X @ w)
    t = np.logaddexp(0.0, mg)
    return np.concatenate([np.maximum(w, 0.0), np.maximum(-w, 0.0), t, np.exp(-t), np.exp(mg - t)])


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_generator_shapes_follow_the_recipe():
    q = I.logistic_exp(2, n_samples=2000, n_features=200, density=0.005)
    N, p = 2000, 200
    assert q["m"] == 7 * N and q["n"] == 2 * p + 3 * N
    assert list(q["cone_types"][:2 * N]) == [I.EXP] * (2 * N) and q["cone_dims"][-1] == N
    X = q["logistic"]["X"]
    assert abs(X.nnz / (N * p) - 0.005) < 0.001
    assert set(np.unique(q["logistic"]["labels"])) == {-1.0, 1.0}
    # nnz: per sample 1 + 1 + (2 nnz(x_i) + 1) + 1 + 2
    assert int(q["row_ptr"][-1]) == 6 * N + 2 * X.nnz
    assert np.isclose(q["logistic"]["lam"], 0.05 * np.abs(X.T @ q["logistic"]["labels"]).max())


def test_lifted_point_is_feasible_with_the_logistic_objective():
    q = I.logistic_exp(4, n_samples=400, n_features=40, density=0.1)
    rng = np.random.default_rng(0)
    K = np.zeros((q["m"], q["n"]))
    for r in range(q["m"]):
        K[r, q["col"][q["row_ptr"][r]:q["row_ptr"][r + 1]]] = q["val"][q["row_ptr"][r]:q["row_ptr"][r + 1]]
    for scale in (0.0, 0.3, 3.0):
        w = scale * rng.standard_normal(40)
        x = lift(q, w)
        s = K @ x - q["h"]
        proj = oracle.proj_cones(s, q["cone_types"], q["cone_dims"])
        assert np.abs(proj - s).max() <= 1e-12 * max(1.0, np.abs(s).max())
        assert abs(q["c"] @ x - logistic_objective(q, w)) <= 1e-12 * abs(logistic_objective(q, w))
        # a loss below the logistic loss leaves the program: the nonnegative row turns negative
        x2 = x.copy()
        N = 400
        x2[80:80 + N] -= 1e-3
        x2[80 + N:80 + 2 * N] = np.exp(-x2[80:80 + N])
        x2[80 + 2 * N:] = np.exp(-q["logistic"]["labels"] * (q["logistic"]["X"] @ w) - x2[80:80 + N])
        s2 = K @ x2 - q["h"]
        assert (s2[6 * N:] < 0.0).all()


@pytest.mark.parametrize("seed", [3, 4])
def test_oracle_optimum_matches_direct_minimisation(seed):
    q = I.logistic_exp(seed, n_samples=60, n_features=8, density=0.3)
    fmin, wmin = logistic_minimum(q)
    s = oracle.Solver(q)
    assert s.run(2_000_000, 1e-8) == oracle.CONVERGED
    x, y = s.solution()
    k = oracle.kkt(q, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1e-8
    assert abs(k["pobj"] - fmin) <= 1e-7 * abs(fmin)
    p = 8
    np.testing.assert_allclose(x[:p] - x[p:2 * p], wmin, atol=1e-3)
