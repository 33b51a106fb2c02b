"""Error paths of the C ABI on the GPU, reached without any device fault: iterates that
overflow to Inf / NaN in ordinary arithmetic (PDCS_ERR_NUMERIC, sticky), a time limit
(PDCS_TIME_LIMIT), and the state calls' argument checks."""
import numpy as np
import pytest

from paper_2505_00311_gb300 import build as B
from paper_2505_00311_gb300 import instances as I
from paper_2505_00311_gb300 import pdcs as P

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def _overflowing_lp(m=200, n=300, seed=4):
    """A finite LP (nonnegative rows only, no root searches) whose right-hand side is so
    large that the first dual step's ||yhat - y||^2 overflows to Inf."""
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(0, 3 * m + 1, 3)
    col = np.concatenate([rng.choice(n, 3, replace=False) for _ in range(m)]).astype(np.int32)
    return {"m": m, "n": n, "row_ptr": row_ptr, "col": col, "val": rng.standard_normal(3 * m),
            "c": rng.standard_normal(n), "h": np.full(m, 1e300), "lb": None, "ub": None,
            "cone_types": np.array([P.CONE_NONNEG]), "cone_dims": np.array([m])}


def test_numeric_error_is_reported_and_sticky():
    g = P.Solver(_overflowing_lp())
    with pytest.raises(P.PdcsError) as e:
        g.solve(1e-6, 1000)
    assert e.value.status == P.ERR_NUMERIC
    assert "NaN" in P.pdcs_last_error(g.ctx)
    with pytest.raises(P.PdcsError) as e:  # the status stays until a new start
        g.solve(1e-6, 1000)
    assert e.value.status == P.ERR_NUMERIC
    assert g.info()["attempts"] <= 64
    # a warm start clears it; the same overflow then recurs
    g.warm_start()
    with pytest.raises(P.PdcsError) as e:
        g.solve(1e-6, 1000)
    assert e.value.status == P.ERR_NUMERIC
    g.close()


def test_time_limit_stops_at_a_check():
    p = I.small_socp(0)
    g = P.Solver(p, time_limit=1e-6, check_period=16)
    st, info = g.solve(1e-14, 1_000_000)
    assert st == P.TIME_LIMIT
    assert 16 <= info["attempts"] < 1_000_000 and info["attempts"] % 16 == 0
    g.close()


def test_set_state_rejects_bad_arguments():
    p = I.small_socp(0)
    g = P.Solver(p)
    st = g.get_state()
    bad = dict(st)
    bad["eta"] = -1.0
    with pytest.raises(P.PdcsError) as e:
        g.set_state(bad)
    assert e.value.status == P.ERR_INVALID
    bad = dict(st)
    bad["x"] = st["x"].copy()
    bad["x"][3] = np.nan
    with pytest.raises(P.PdcsError) as e:
        g.set_state(bad)
    assert e.value.status == P.ERR_INVALID
    bad = dict(st)
    bad["status"] = 7
    with pytest.raises(P.PdcsError) as e:
        g.set_state(bad)
    assert e.value.status == P.ERR_INVALID
    g.close()
