"""The learned starting point of the exponential-cone root search: the GPU forward /
backward kernels against the FP64 reference network, training on pairs the plain
projector computes, and what the trained network gains over the cold start (the
projection itself is unchanged and stays equal to the oracle's to 1e-12)."""
import numpy as np
import pytest

import oracle
from oracle import exp_mlp as M
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def _inputs(seed, n):
    """Projection workload of the paper's exp-cone timing (3-vectors N(0, 1)), with random
    positive scales exp(N(0, 0.5^2)) per coordinate."""
    rng = np.random.default_rng(seed)
    return rng.normal(size=(n, 3)), np.exp(rng.normal(0.0, 0.5, (n, 3)))


@pytest.fixture(scope="module")
def trained():
    v, d = _inputs(11, 400_000)
    X, t = P.exp_mlp_dataset(v, d)
    w0 = P.exp_mlp_init(0)
    w, trace = P.exp_mlp_train(X, t, w0, steps=4000, batch=4096, lr=2e-3, seed=5)
    return X, t, w0, w, trace


def test_gpu_loss_and_gradient_match_the_reference_network():
    rng = np.random.default_rng(3)
    w = P.exp_mlp_init(1)
    X = rng.normal(size=(1000, M.IN)).astype(np.float32)
    t = (3.0 * rng.normal(size=1000)).astype(np.float32)
    loss, g = P.exp_mlp_loss_grad(X, t, w)
    lo, go = M.loss_grad(w.astype(np.float64), X.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()


def test_dataset_pairs_are_the_plain_search_roots(trained):
    X, t, _, _, _ = trained
    assert len(t) > 50_000 and np.all(np.isfinite(t)) and np.all(np.isfinite(X))
    # features: a unit direction, two log scale ratios, one branch flag
    np.testing.assert_allclose(np.linalg.norm(X[:, :3], axis=1), 1.0, rtol=1e-5)
    np.testing.assert_array_equal(X[:, 5:].sum(axis=1), 1.0)


def test_training_fits_the_roots(trained):
    X, t, w0, w, trace = trained
    l0, _ = P.exp_mlp_loss_grad(X, t, w0)
    l1, _ = P.exp_mlp_loss_grad(X, t, w)
    assert np.all(np.isfinite(trace))
    assert l1 < 0.1 * l0, (l0, l1)
    assert l1 < 0.5 * float(np.var(t)), (l1, np.var(t))  # far better than the mean guess


def test_trained_network_saves_root_search_evaluations(trained):
    _, _, _, w, _ = trained
    v, d = _inputs(12, 100_000)  # fresh inputs
    out0, ev0 = P.exp_proj_stats(v, d, None)
    out1, ev1 = P.exp_proj_stats(v, d, w)
    case4 = ev0.sum(axis=1) > 0
    assert case4.sum() > 10_000
    scale = np.maximum(1.0, np.abs(v).max(axis=1))
    # the network moves only the starting point: same projection to the search's tolerance
    assert (np.abs(out1 - out0).max(axis=1) / scale).max() <= 1e-12
    sample = np.flatnonzero(case4)[:1500]
    for i in sample:
        ref = oracle.proj_exp(v[i], d[i])
        assert np.abs(out1[i] - ref).max() <= 1e-12 * scale[i]
    e32_cold, e32_mlp = ev0[case4, 0].mean(), ev1[case4, 0].mean()
    e64_cold, e64_mlp = ev0[case4, 1].mean(), ev1[case4, 1].mean()
    print("evaluations of h per case-4 cone (FP32, FP64): cold %.2f, %.2f; learned start %.2f, %.2f"
          % (e32_cold, e64_cold, e32_mlp, e64_mlp))
    # the network saves Newton steps; the bracket set-up (the sign at the midpoint of a
    # finite interval or the growth of an infinite one, and the endpoint value) stays
    assert e32_mlp <= e32_cold - 0.2
    assert e64_mlp <= e64_cold + 0.05  # FP64 work not increased


def test_solver_with_the_network_reaches_the_same_solution(trained):
    _, _, _, w, _ = trained
    p = I.scaled_mixed_cone(1, 0.01)
    g = P.Solver(p, exp_mlp=w)
    st, info = g.solve(1e-6, 400_000)
    assert st == P.OK, info
    x, y = g.solution()
    k = oracle.kkt(p, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1.01e-6
    assert abs(k["pobj"] - p["obj_star"]) <= 1e-5 * (1 + abs(p["obj_star"]))
    g.close()
