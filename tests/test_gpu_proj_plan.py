"""The projection plan (pdcs_proj_plan_*): cone layout built once, runs that only enqueue
kernels, SOC strategy by dimension (warp, or a team of blocks of a cooperative launch).
Against the oracle's projections block by block (1e-12 of the block norm), primal and
dual, D = I and random D, cone lists that mix every strategy, two runs in a row."""
import numpy as np
import pytest

import oracle
from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()
    oracle.build()


def _layout(rng, kind):
    if kind == "mixed":  # every strategy: scalar blocks, small and mid SOC (warp), large SOC / RSOC (teams), exp
        types = [0, 1, 2, 3, 4, 2, 1, 3, 2, 4, 4, 2]
        dims = [5, 7, 40, 300, 3, 5000, 9, 70_001, 200_000, 3, 3, 1_500_000]
    else:  # many equal large cones: several waves of teams
        types = [2] * 40
        dims = [60_000] * 40
    return np.array(types, np.int32), np.array(dims, np.int64)


def _inputs(rng, types, dims, scaled):
    m = int(dims.sum())
    v = rng.standard_normal(m)
    o = 0
    for t, k in zip(types, dims):  # SOC first entries where the projection is a genuine root search
        if t in (2, 3) and k > 2:
            v[o] = rng.uniform(-1.0, 1.0) * np.linalg.norm(v[o + 1:o + k])
        o += k
    d = None
    if scaled:
        d = np.exp(rng.normal(0, 0.5, m))
        o = 0
        for t, k in zip(types, dims):
            if t == 3:
                d[o + 1] = d[o]
            o += k
    return v, d


@pytest.mark.parametrize("kind", ["mixed", "waves"])
@pytest.mark.parametrize("scaled", [False, True])
@pytest.mark.parametrize("dual", [0, 1])
def test_plan_matches_oracle(kind, scaled, dual):
    import torch
    rng = np.random.default_rng(3 + 2 * scaled + dual + 10 * (kind == "waves"))
    types, dims = _layout(rng, kind)
    m = int(dims.sum())
    stream = torch.cuda.current_stream().cuda_stream
    plan = P.ProjPlan(m, types, dims, stream)
    for rep in range(2):
        v, d = _inputs(rng, types, dims, scaled)
        tv = torch.tensor(v, dtype=torch.float64, device="cuda")
        td = None if d is None else torch.tensor(d, dtype=torch.float64, device="cuda")
        out = torch.full_like(tv, float("nan"))
        plan.run(tv.data_ptr(), 0 if td is None else td.data_ptr(), dual, out.data_ptr(), stream)
        assert plan.check(stream) == P.OK
        got = out.cpu().numpy()
        ref = oracle.proj_cones(v, types, dims, d, dual=bool(dual))
        o = 0
        for t, k in zip(types, dims):
            blk = slice(o, o + k)
            scale = max(np.linalg.norm(v[blk]), 1e-300)
            assert np.linalg.norm(got[blk] - ref[blk]) <= 1e-12 * scale, (rep, t, k)
            o += k
    plan.close()


def test_plan_in_place_and_rejects_bad_lists():
    import torch
    rng = np.random.default_rng(1)
    types, dims = np.array([2, 1], np.int32), np.array([10_000, 5], np.int64)
    m = int(dims.sum())
    v, _ = _inputs(rng, types, dims, False)
    ref = oracle.proj_cones(v, types, dims, None, dual=False)
    tv = torch.tensor(v, dtype=torch.float64, device="cuda")
    plan = P.ProjPlan(m, types, dims)
    plan.run(tv.data_ptr(), 0, 0, tv.data_ptr())
    assert plan.check() == P.OK
    assert np.linalg.norm(tv.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(v)
    plan.close()
    with pytest.raises(P.PdcsError):
        P.ProjPlan(m + 1, types, dims)
    with pytest.raises(P.PdcsError):
        P.ProjPlan(6, np.array([4, 4], np.int32), np.array([3, 2], np.int64))
