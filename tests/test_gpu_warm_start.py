"""Learned warm start of a parametric program family: a network maps a summary of an
instance's returns to its dual solution and primal weight; solves started from the
prediction (x = 0, y0, omega0) are compared with cold starts at the same tolerance.
The network is trained on the GPU by the library's kernels on solutions the solver
computes (a batch), and its gradients are checked against the FP64 reference."""
import numpy as np
import pytest

import oracle
from oracle import mlp as N
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    oracle.build()


def test_gpu_network_loss_and_gradient_match_the_reference():
    sizes = [17, 64, 48, 23]
    rng = np.random.default_rng(2)
    W = P.mlp_init(sizes, 3)
    assert W.size == P.mlp_params(sizes)
    X = rng.normal(size=(300, sizes[0])).astype(np.float32)
    T = rng.normal(size=(300, sizes[-1])).astype(np.float32)
    loss, g = P.mlp_loss_grad(sizes, X, T, W)
    lo, go = N.loss_grad(sizes, W.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert abs(loss - lo) <= 1e-5 * lo
    assert np.abs(g - go).max() <= 1e-4 * np.abs(go).max()
    Y = P.mlp_forward(sizes, X, W)
    np.testing.assert_allclose(Y, N.forward(sizes, W.astype(np.float64), X), rtol=1e-4, atol=1e-5)


def _bf16(a):
    """Round to the nearest BF16 (ties to even), in FP64: the top 16 bits of the FP32 value."""
    f = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    f = (f + 0x7FFF + ((f >> 16) & 1)) & 0xFFFF0000
    return f.astype(np.uint32).view(np.float32).astype(np.float64)


def test_bf16_tensor_core_forward_matches_the_reference():
    """pdcs_mlp_forward_bf16 (mma.sync m16n8k16 tiles, BF16 operands, FP32 accumulation) on the
    warm-start network's shape and on ragged sizes (rows, inputs and outputs that are not
    multiples of the tile): against the FP64 forward of oracle/mlp.py with the same BF16
    roundings of the rows, weights and hidden activations, within 1e-4 of the scale of each
    layer's products, and against the FP32 forward within the BF16 rounding."""
    rng = np.random.default_rng(4)
    for sizes, n in (([17, 256, 256, 23], 1000), ([9, 40, 13], 37), ([5, 3], 1)):
        W = P.mlp_init(sizes, 5).astype(np.float32)
        X = rng.normal(size=(n, sizes[0])).astype(np.float32)
        Y = P.mlp_forward_bf16(sizes, X, W)
        # reference: layer by layer, the products of BF16-rounded operands in FP64
        h = X.astype(np.float64)
        off = 0
        scale = 0.0
        for l in range(len(sizes) - 1):
            din, dout = sizes[l], sizes[l + 1]
            Wl = W[off:off + din * dout].reshape(dout, din).astype(np.float64)
            off += din * dout
            bl = W[off:off + dout].astype(np.float64)
            off += dout
            prod = _bf16(h) @ _bf16(Wl).T
            scale = np.abs(_bf16(h)) @ np.abs(_bf16(Wl)).T
            h = prod + bl
            if l + 1 < len(sizes) - 1:
                h = np.maximum(h, 0.0)
        # the last layer's inputs differ from the reference only by FP32 sums (and, rarely, by
        # the BF16 rounding of an activation they moved across a tie)
        assert np.max(np.abs(Y - h) / (scale + 1e-30)) <= 1e-2
        assert np.median(np.abs(Y - h) / (scale + 1e-30)) <= 1e-5
        Y32 = P.mlp_forward(sizes, X, W)
        assert np.max(np.abs(Y - Y32) / (scale + 1e-30)) <= 4e-2


FAM_ASSETS, FAM_FACTORS = 400, 10
SIZES = [FAM_FACTORS + 7, 256, 256, 1 + 2 * FAM_FACTORS + 2]


def _solve_all(fam, seeds, warm=None):
    """Solves the instances in one batch; warm: per instance (y0, omega0) or None."""
    solvers = []
    for k, sd in enumerate(seeds):
        s = P.Solver(I.portfolio_socp(fam, I.portfolio_mu(fam, sd)), batch_blocks=4)
        if warm is not None:
            s.warm_start(None, warm[k][0], warm[k][1])
        solvers.append(s)
    b = P.Batch(solvers)
    st, nconv = b.solve(1e-6, 200_000)
    res = [(s.solution(), s.info()) for s in solvers]
    b.close()
    for s in solvers:
        s.close()
    return nconv, res


@pytest.fixture(scope="module")
def family_model():
    fam = I.portfolio_family(0, FAM_ASSETS, FAM_FACTORS)
    train = list(range(160))
    nconv, res = _solve_all(fam, train)
    assert nconv == len(train)
    X = np.stack([I.portfolio_features(fam, I.portfolio_mu(fam, sd)) for sd in train])
    Y = np.stack([np.concatenate([[np.log(info["omega"])], y]) for (x, y), info in res])
    mu_y, sd_y = Y.mean(axis=0), Y.std(axis=0) + 1e-12
    mu_x, sd_x = X.mean(axis=0), X.std(axis=0) + 1e-12
    W0 = P.mlp_init(SIZES, 0)
    W, trace = P.mlp_train(SIZES, (X - mu_x) / sd_x, (Y - mu_y) / sd_y, W0, steps=3000, batch=64, lr=1e-3, seed=7)
    return fam, W, (mu_x, sd_x, mu_y, sd_y), trace, res


def test_warm_start_network_fits_the_training_solutions(family_model):
    _, _, _, trace, _ = family_model
    assert np.all(np.isfinite(trace))
    assert trace[-200:].mean() < 0.1 * trace[:20].mean()


def test_learned_warm_start_saves_evaluations(family_model):
    fam, W, (mu_x, sd_x, mu_y, sd_y), _, _ = family_model
    held = list(range(1000, 1024))
    X = np.stack([I.portfolio_features(fam, I.portfolio_mu(fam, sd)) for sd in held])
    pred = P.mlp_forward(SIZES, (X - mu_x) / sd_x, W) * sd_y + mu_y
    warm = [(p[1:].astype(np.float64), float(np.exp(p[0]))) for p in pred]
    n0, cold = _solve_all(fam, held)
    n1, hot = _solve_all(fam, held, warm)
    assert n0 == n1 == len(held)
    for sd, ((x, y), info) in zip(held, hot):
        p = I.portfolio_socp(fam, I.portfolio_mu(fam, sd))
        k = oracle.kkt(p, x, y)
        assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1.01e-6
    e_cold = np.mean([info["attempts"] for _, info in cold])
    e_hot = np.mean([info["attempts"] for _, info in hot])
    print("evaluations to 1e-6: cold %.0f, learned warm start %.0f" % (e_cold, e_hot))
    assert e_hot < e_cold
