"""Dual-exponential-cone row blocks (PDCS_CONE_EXP_DUAL: rows in K_exp^*, the dual-cone row
blocks of the problem of Sec. 2) against the FP64 oracle: projections onto D K_exp^* and its
dual D^{-1} K_exp through both projection entry points, one PDHG evaluation from the
oracle's states, and a solve of a known-optimum program judged by the oracle's KKT
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


def _layout(rng, n_blocks):
    types, dims = [], []
    for _ in range(n_blocks):
        t = int(rng.choice([0, 1, 2, 4, 5, 5]))
        types.append(t)
        dims.append({0: 3, 1: 4, 2: int(rng.integers(2, 40)), 4: 3, 5: 3}[t])
    return np.array(types, np.int32), np.array(dims, np.int64)


@pytest.mark.parametrize("dual", [0, 1])
@pytest.mark.parametrize("scaled", [False, True])
def test_exp_dual_projections_match_the_oracle(dual, scaled):
    import torch
    rng = np.random.default_rng(21 + dual + 2 * scaled)
    types, dims = _layout(rng, 3000)
    m = int(dims.sum())
    v = rng.standard_normal(m) * np.exp(rng.normal(0, 1.5, m))
    d = np.exp(rng.normal(0, 0.8, m)) if scaled else None
    ref = oracle.proj_cones(v, types, dims, d, dual=bool(dual))
    tv = torch.tensor(v, dtype=torch.float64, device="cuda")
    td = None if d is None else torch.tensor(d, dtype=torch.float64, device="cuda")
    dp = 0 if td is None else td.data_ptr()
    stream = torch.cuda.current_stream().cuda_stream
    a = torch.empty_like(tv)
    P.pdcs_proj_cones_device(tv.data_ptr(), dp, m, types, dims, dual, a.data_ptr(), stream)
    plan = P.ProjPlan(m, types, dims, stream)
    b = torch.empty_like(tv)
    plan.run(tv.data_ptr(), dp, dual, b.data_ptr(), stream)
    assert plan.check(stream) == P.OK
    plan.close()
    for got in (a.cpu().numpy(), b.cpu().numpy()):
        o = 0
        for t, k in zip(types, dims):
            blk = slice(o, o + k)
            assert np.linalg.norm(got[blk] - ref[blk]) <= RTOL * max(np.linalg.norm(v[blk]), 1e-300), (t, k)
            o += k


def test_one_evaluation_with_exp_dual_blocks():
    """One evaluation from the oracle's states after 0, 64 and 300 evaluations of the program
    with EXP and EXP_DUAL blocks: every role within 1e-12."""
    from parity_helpers import one_evaluation
    p = I.dual_exp_program(3)
    o = oracle.Solver(p, check_period=64)
    g = P.Solver(p, check_period=64)
    done = 0
    for start in [0, 64, 300]:
        o.run(start - done)
        err, acc = one_evaluation(p, g, o)
        done = start + 1
        assert acc[0] == acc[1] and max(err.values()) <= RTOL, (start, err)
    g.close()


def test_solve_with_exp_dual_blocks_reaches_the_known_optimum():
    p = I.dual_exp_program(3)
    g = P.Solver(p)
    st, info = g.solve(1e-6, 1_000_000)
    assert st == P.OK
    x, y = g.solution()
    k = oracle.kkt(p, x, y)
    assert max(k["err_p"], k["err_d"], k["err_gap"]) <= 1e-6, k
    assert k["pobj"] == pytest.approx(p["obj_star"], rel=1e-4, abs=1e-4)
    g.close()
