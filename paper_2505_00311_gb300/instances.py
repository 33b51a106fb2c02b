"""Seeded synthetic conic programs with a known optimal primal-dual pair.

This module only draws inputs; it holds none of the solver's arithmetic and is
shared by the tests, the benchmark and the smoke check.  Every generator uses
numpy's PCG64 through ``np.random.default_rng(seed)``.

Known-optimum construction (used for the mixed-cone programs):
pick x* >= 0 and lambda* >= 0 with complementary supports, and per cone a
complementary slack/dual pair s* in C, y* in C* with <s*, y*> = 0:
  - zero rows:    s* = 0, y* ~ N(0, 1);
  - nonneg rows:  half with s* > 0, y* = 0; half with s* = 0, y* > 0;
  - SOC blocks:   a third on the boundary, s* = a (1, u), y* = b (1, -u), ||u|| = 1;
                  a third with s* interior, y* = 0; a third with y* interior, s* = 0;
  - exp blocks:   s* = a (rho, 1, e^rho), y* = b (-1, rho - 1, e^-rho) (orthogonal for
                  every rho, as in the proof of Theorem 3), or one side interior and
                  the other zero.
Then c = K'y* + lambda* and h = K x* - s*; with l = 0, u = +inf every KKT
residual of (x*, y*) vanishes and the optimal value is c'x* = h'y*.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

ZERO, NONNEG, SOC, RSOC, EXP, EXP_DUAL = 0, 1, 2, 3, 4, 5


def _unique_cols(rng, row_ptr, n):
    """Uniform column indices without repeats inside a row, sorted per row."""
    m = row_ptr.size - 1
    nnz = int(row_ptr[-1])
    rows = np.repeat(np.arange(m, dtype=np.int64), np.diff(row_ptr))
    cols = rng.integers(0, n, size=nnz, dtype=np.int64)
    for _ in range(64):
        key = rows * n + cols
        order = np.argsort(key, kind="stable")
        cols = cols[order]
        key = key[order]
        dup = np.zeros(nnz, dtype=bool)
        dup[1:] = key[1:] == key[:-1]
        if not dup.any():
            break
        cols[dup] = rng.integers(0, n, size=int(dup.sum()), dtype=np.int64)
    return cols.astype(np.int32)


def _soc_pair(rng, dim):
    """(s*, y*) for one SOC block of size dim (dim >= 2)."""
    kind = rng.integers(0, 3)
    s = np.zeros(dim)
    y = np.zeros(dim)
    if kind == 0:  # both on the boundary, orthogonal
        u = rng.standard_normal(dim - 1)
        u /= np.linalg.norm(u)
        a, b = rng.uniform(0.5, 1.5, 2)
        s[0], s[1:] = a, a * u
        y[0], y[1:] = b, -b * u
    elif kind == 1:  # s* interior
        w = rng.standard_normal(dim - 1)
        s[0], s[1:] = np.linalg.norm(w) + rng.uniform(0.1, 1.0), w
    else:  # y* interior
        w = rng.standard_normal(dim - 1)
        y[0], y[1:] = np.linalg.norm(w) + rng.uniform(0.1, 1.0), w
    return s, y


def _exp_pair(rng):
    kind = rng.integers(0, 3)
    if kind == 0:
        rho = rng.uniform(-2.0, 2.0)
        a, b = rng.uniform(0.5, 1.5, 2)
        return a * np.array([rho, 1.0, np.exp(rho)]), b * np.array([-1.0, rho - 1.0, np.exp(-rho)])
    if kind == 1:  # s* interior of K_exp: s > 0, t > s exp(r / s)
        r, s_ = rng.uniform(-1.0, 1.0), rng.uniform(0.5, 1.5)
        t = s_ * np.exp(r / s_) * (1.0 + rng.uniform(0.1, 1.0))
        return np.array([r, s_, t]), np.zeros(3)
    r, s_ = -rng.uniform(0.5, 1.5), rng.uniform(-1.0, 1.0)  # y* interior of K_exp^*
    t = (-r / np.e) * np.exp(s_ / r) * (1.0 + rng.uniform(0.1, 1.0))
    return np.zeros(3), np.array([r, s_, t])


def _primal_pair(rng, n, lb, ub):
    """x* in [l, u] and lambda* in Lambda (eq. defn_Lambda1) with l'lam^+ - u'lam^- = lam'x*."""
    x = np.zeros(n)
    lam = np.zeros(n)
    if lb is None and ub is None:
        pos = rng.random(n) < 0.5
        x[pos] = rng.uniform(0.1, 1.0, int(pos.sum()))
        lam[~pos] = rng.uniform(0.1, 1.0, int((~pos).sum()))
        return x, lam
    for j in range(n):
        lf, uf = np.isfinite(lb[j]), np.isfinite(ub[j])
        opts = ["in"] + (["lo"] if lf else []) + (["up"] if uf else [])
        k = opts[rng.integers(0, len(opts))]
        if k == "lo":
            x[j], lam[j] = lb[j], rng.uniform(0.1, 1.0)
        elif k == "up":
            x[j], lam[j] = ub[j], -rng.uniform(0.1, 1.0)
        else:
            a = lb[j] if lf else (ub[j] - 2.0 if uf else -1.0)
            b = ub[j] if uf else a + 2.0
            x[j] = a + (b - a) * rng.uniform(0.2, 0.8)
    return x, lam


def _finish(rng, m, n, row_ptr, cols, vals, cone_types, cone_dims, name, lb=None, ub=None):
    """Draw (x*, lambda*, s*, y*) and set c, h so that (x*, y*) is optimal."""
    K = sp.csr_matrix((vals, cols, row_ptr), shape=(m, n))
    x, lam = _primal_pair(rng, n, lb, ub)
    s = np.zeros(m)
    y = np.zeros(m)
    o = 0
    for t, d in zip(cone_types, cone_dims):
        d = int(d)
        if t == ZERO:
            y[o:o + d] = rng.standard_normal(d)
        elif t == NONNEG:
            half = rng.random(d) < 0.5
            s[o:o + d][half] = rng.uniform(0.1, 1.0, int(half.sum()))
            y[o:o + d][~half] = rng.uniform(0.1, 1.0, int((~half).sum()))
        elif t == SOC:
            if d == 1:
                s[o] = rng.uniform(0.1, 1.0)
            else:
                s[o:o + d], y[o:o + d] = _soc_pair(rng, d)
        elif t == RSOC:  # K_rsoc = Q K_soc, Q = [[1, 1], [1, -1]] / sqrt2 (+) I, orthogonal
            ss, yy = _soc_pair(rng, d)
            for v in (ss, yy):
                a, b = v[0], v[1]
                v[0], v[1] = (a + b) / np.sqrt(2.0), (a - b) / np.sqrt(2.0)
            s[o:o + d], y[o:o + d] = ss, yy
        elif t == EXP:
            s[o:o + 3], y[o:o + 3] = _exp_pair(rng)
        elif t == EXP_DUAL:  # the block is K_exp^*: the pair with the roles of the cones swapped
            y[o:o + 3], s[o:o + 3] = _exp_pair(rng)
        else:
            raise ValueError("unsupported cone in the known-optimum construction")
        o += d
    c = K.T @ y + lam
    h = K @ x - s
    return {
        "name": name, "m": m, "n": n, "row_ptr": row_ptr, "col": cols, "val": vals,
        "c": c, "h": h, "lb": lb, "ub": ub,
        "cone_types": np.asarray(cone_types, dtype=np.int32),
        "cone_dims": np.asarray(cone_dims, dtype=np.int64),
        "x_star": x, "y_star": y, "s_star": s, "lambda_star": lam, "obj_star": float(c @ x),
    }


def small_socp(seed: int = 0, n: int = 2000, m: int = 1000, row_nnz: int = 20,
               n_nonneg: int = 500, n_soc: int = 50, soc_dim: int = 10):
    """Random sparse SOCP: n = 2,000, m = 1,000, 20 nonzeros per row (uniform columns,
    N(0,1) values), C = 500 nonnegative rows + 50 SOC(10), x >= 0, known optimum."""
    assert n_nonneg + n_soc * soc_dim == m
    rng = np.random.default_rng(seed)
    row_ptr = np.arange(m + 1, dtype=np.int64) * row_nnz
    cols = _unique_cols(rng, row_ptr, n)
    vals = rng.standard_normal(row_ptr[-1])
    types = [NONNEG] + [SOC] * n_soc
    dims = [n_nonneg] + [soc_dim] * n_soc
    return _finish(rng, m, n, row_ptr, cols, vals, types, dims, "small_socp")


def mixed_cone(seed: int = 1, n: int = 1_000_000, m: int = 500_000, nnz: int = 10_000_000,
               n_nonneg: int = 200_000, soc_rows: int = 200_000, n_exp: int = 20_000,
               soc_dim_range=(4, 64), scalar_chunk: int = 1000):
    """Large mixed-cone LP/SOCP/exp program: row degrees clip(round(LogNormal(2.5, 1)), 2, 200)
    rescaled to ~nnz in total, N(0,1) values, 200k nonnegative rows, SOC blocks of
    dimension U{4..64} filling 200k rows, 20k exponential cones, the remaining rows zero
    cones; block order shuffled; known optimum."""
    n_zero = m - n_nonneg - soc_rows - 3 * n_exp
    assert n_zero >= 0
    rng = np.random.default_rng(seed)
    deg = np.clip(np.round(rng.lognormal(2.5, 1.0, m)), 2, 200)
    deg = np.clip(np.round(deg * (nnz / deg.sum())), 2, 200).astype(np.int64)
    deg = np.minimum(deg, n)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(deg, out=row_ptr[1:])
    cols = _unique_cols(rng, row_ptr, n)
    vals = rng.standard_normal(int(row_ptr[-1]))
    soc_dims = []
    left = soc_rows
    lo, hi = soc_dim_range
    while left > 0:
        d = int(rng.integers(lo, hi + 1))
        if left - d < lo and left - d != 0:
            d = left
        soc_dims.append(d)
        left -= d
    blocks = []
    for k in range(0, n_zero, scalar_chunk):
        blocks.append((ZERO, min(scalar_chunk, n_zero - k)))
    for k in range(0, n_nonneg, scalar_chunk):
        blocks.append((NONNEG, min(scalar_chunk, n_nonneg - k)))
    blocks += [(SOC, d) for d in soc_dims]
    blocks += [(EXP, 3)] * n_exp
    order = rng.permutation(len(blocks))
    types = [blocks[i][0] for i in order]
    dims = [blocks[i][1] for i in order]
    return _finish(rng, m, n, row_ptr, cols, vals, types, dims, "mixed_cone")


def mixed_cone_literal(seed: int = 1):
    """The mixed-cone recipe with the literal cone counts: 50k SOC blocks of dimension
    U{4..64} (about 1.7M rows), 200k nonnegative rows, 20k exp cones and 40k zero rows, so
    m = 2,000,000; n = 1,000,000 and ~41M nonzeros (mean row degree 20.5)."""
    return mixed_cone(seed=seed, n=1_000_000, m=2_000_000, nnz=41_000_000, n_nonneg=200_000,
                      soc_rows=1_700_000, n_exp=20_000)


def scaled_mixed_cone(seed: int = 1, scale: float = 0.01):
    """The mixed-cone program at a fraction of its size (same recipe)."""
    n = int(1_000_000 * scale)
    m = int(500_000 * scale)
    return mixed_cone(seed=seed, n=n, m=m, nnz=int(10_000_000 * scale),
                      n_nonneg=int(200_000 * scale), soc_rows=int(200_000 * scale),
                      n_exp=int(20_000 * scale), scalar_chunk=max(1, int(1000 * scale)))


def dual_exp_program(seed: int = 3, n: int = 800, row_nnz: int = 10):
    """Random sparse program with exponential-cone blocks and dual-exponential-cone blocks
    (rows constrained to K_exp^*, the dual-cone row blocks of the problem of Sec. 2) beside
    zero, nonnegative and SOC rows: 100 zero, 200 nonneg, 20 SOC(5), 30 EXP, 70 EXP_DUAL
    (m = 700), 10 uniform columns per row, N(0,1) values, known optimum (an EXP_DUAL block
    takes the exp pair with s* in K_exp^* and y* in K_exp)."""
    rng = np.random.default_rng(seed)
    types = [ZERO, NONNEG] + [SOC] * 20 + [EXP] * 30 + [EXP_DUAL] * 70
    dims = [100, 200] + [5] * 20 + [3] * 30 + [3] * 70
    order = rng.permutation(len(types) - 2) + 2  # interleave the cone blocks after the scalar rows
    types = types[:2] + [types[k] for k in order]
    dims = dims[:2] + [dims[k] for k in order]
    m = int(sum(dims))
    row_ptr = np.arange(m + 1, dtype=np.int64) * row_nnz
    cols = _unique_cols(rng, row_ptr, n)
    vals = rng.standard_normal(int(row_ptr[-1]))
    return _finish(rng, m, n, row_ptr, cols, vals, types, dims, "dual_exp_program")


def primal_cone_program(seed: int = 4, n_before: int = 300, pcone_dims=(5, 40, 2, 120, 9),
                        pcone_types=None, n_after: int = 200, m: int = 400, row_nnz: int = 8):
    """A program with primal cone blocks x2 in K_p (Sec. 2, eq. prob_cp with n2 > 0) and a known
    optimum: variables [n_before box | the cone blocks | n_after box], the box variables in
    [0, +inf), the cone variables free of bounds and grouped into SOC / RSOC blocks (types
    alternate SOC, RSOC unless given); rows: a quarter zero, a quarter nonneg, the rest SOC
    blocks of 10 rows; row_nnz N(0, 1) entries per row at uniform columns.  The optimal pair
    follows the construction of the module docstring, with each cone block of x* and its reduced
    cost lambda* drawn as a complementary (s*, y*) pair of that cone (K_p^* = K_p)."""
    rng = np.random.default_rng(seed)
    pcone_dims = [int(d) for d in pcone_dims]
    if pcone_types is None:
        pcone_types = [SOC if k % 2 == 0 else RSOC for k in range(len(pcone_dims))]
    if any(d < (2 if t == RSOC else 1) for t, d in zip(pcone_types, pcone_dims)):
        raise ValueError("an SOC block needs at least 1 variable, an RSOC block at least 2")
    n_pc = sum(pcone_dims)
    n = n_before + n_pc + n_after
    row_ptr = np.arange(m + 1, dtype=np.int64) * row_nnz
    cols = _unique_cols(rng, row_ptr, n)
    vals = rng.standard_normal(m * row_nnz)
    mz, mn = m // 4, m // 4
    n_soc = (m - mz - mn) // 10
    types = [ZERO, NONNEG] + [SOC] * n_soc
    dims = [mz, mn + (m - mz - mn - 10 * n_soc)] + [10] * n_soc
    lb = np.zeros(n)
    ub = np.full(n, np.inf)
    lb[n_before:n_before + n_pc] = -np.inf
    p = _finish(rng, m, n, row_ptr, cols, vals, types, dims, "primal_cone_program", lb=lb, ub=ub)
    x, lam = p["x_star"], p["lambda_star"]
    o = n_before
    for t, d in zip(pcone_types, pcone_dims):
        xs, ls = (_soc_pair(rng, d) if d >= 2 else (np.array([rng.uniform(0.1, 1.0)]), np.zeros(1)))
        if t == RSOC:
            for v in (xs, ls):
                a, b = v[0], v[1]
                v[0], v[1] = (a + b) / np.sqrt(2.0), (a - b) / np.sqrt(2.0)
        x[o:o + d], lam[o:o + d] = xs, ls
        o += d
    K = sp.csr_matrix((vals, cols, row_ptr), shape=(m, n))
    p["c"] = K.T @ p["y_star"] + lam
    p["h"] = K @ x - p["s_star"]
    p["obj_star"] = float(p["c"] @ x)
    p["pcone_types"] = np.asarray(pcone_types, dtype=np.int32)
    p["pcone_dims"] = np.asarray(pcone_dims, dtype=np.int64)
    p["pcone_start"] = n_before
    return p


def edge_cases(seed: int = 5, m: int = 40, n: int = 30):
    """Small program with every cone kind (zero, nonneg, RSOC, SOC, exp), empty rows,
    two empty columns, finite boxes, one-sided bounds and free variables; known optimum."""
    rng = np.random.default_rng(seed)
    degs = [0 if i % 7 == 3 else int(rng.integers(1, 6)) for i in range(m)]
    row_ptr = np.zeros(m + 1, np.int64)
    row_ptr[1:] = np.cumsum(degs)
    cols = np.concatenate([np.sort(rng.choice(n - 2, size=k, replace=False)) for k in degs]).astype(np.int32)
    vals = rng.standard_normal(int(row_ptr[-1]))
    types = [ZERO, NONNEG, RSOC, SOC, EXP, RSOC]
    dims = [5, 10, 6, 12, 3, 4]
    assert sum(dims) == m
    kind = rng.integers(0, 4, n)  # 0 box, 1 lower only, 2 upper only, 3 free
    lb = np.where((kind == 0) | (kind == 1), -rng.uniform(0.0, 1.0, n), -np.inf)
    ub = np.where((kind == 0) | (kind == 2), rng.uniform(0.5, 1.5, n), np.inf)
    return _finish(rng, m, n, row_ptr, cols, vals, types, dims, "edge_cases", lb=lb, ub=ub)


def lasso_socp(seed: int = 0, n: int = 200, m: int | None = None, lam: float | None = None):
    """Lasso min ||A x - b||^2 + lam ||x||_1 as the SOCP of the paper's App. C (variables
    w, r, y (m), x1, x2 (n each), x = x1 - x2): w = 1 and y = A(x1 - x2) - b as zero rows,
    (w, r, y) in the rotated SOC ||y||^2 <= 2 w r, objective 2 r + lam 1'(x1 + x2), x1, x2 >= 0,
    w, r, y free.  Data (batched-workload recipe): m = n / 2, A dense N(0, 1), a ground truth
    with 5 % nonzero N(0, 1) entries, b = A x~ + 0.01 N(0, 1), lam ~ U[0.01, 1].  No known
    optimum: solutions are checked by the KKT evaluator."""
    rng = np.random.default_rng(seed)
    m = max(1, n // 2) if m is None else m
    A = rng.standard_normal((m, n))
    xt = np.zeros(n)
    nz = rng.random(n) < 0.05
    xt[nz] = rng.standard_normal(int(nz.sum()))
    b = A @ xt + 0.01 * rng.standard_normal(m)
    lam = float(rng.uniform(0.01, 1.0)) if lam is None else float(lam)
    nv = 2 + m + 2 * n
    iw, ir, iy, ix1, ix2 = 0, 1, 2, 2 + m, 2 + m + n
    rows, cols, vals = [], [], []
    # zero rows: w = 1, then y - A x1 + A x2 = -b
    rows.append([0]); cols.append([iw]); vals.append([1.0])
    for i in range(m):
        r = 1 + i
        rows.append(np.full(1 + 2 * n, r))
        cols.append(np.concatenate([[iy + i], ix1 + np.arange(n), ix2 + np.arange(n)]))
        vals.append(np.concatenate([[1.0], -A[i], A[i]]))
    # rotated SOC rows (w, r, y)
    o = 1 + m
    rows.append(o + np.arange(m + 2)); cols.append(np.concatenate([[iw, ir], iy + np.arange(m)]))
    vals.append(np.ones(m + 2))
    R = np.concatenate([np.asarray(x) for x in rows])
    C = np.concatenate([np.asarray(x) for x in cols])
    V = np.concatenate([np.asarray(x, dtype=float) for x in vals])
    M = sp.csr_matrix((V, (R, C)), shape=(2 * m + 3, nv))
    M.sort_indices()
    c = np.zeros(nv)
    c[ir] = 2.0
    c[ix1:] = lam
    h = np.zeros(2 * m + 3)
    h[0] = 1.0
    h[1:1 + m] = -b
    lb = np.full(nv, -np.inf)
    lb[ix1:] = 0.0
    ub = np.full(nv, np.inf)
    return {"name": "lasso_socp", "m": 2 * m + 3, "n": nv, "row_ptr": M.indptr.astype(np.int64),
            "col": M.indices.astype(np.int32), "val": M.data, "c": c, "h": h, "lb": lb, "ub": ub,
            "cone_types": np.asarray([ZERO, RSOC], dtype=np.int32),
            "cone_dims": np.asarray([1 + m, m + 2], dtype=np.int64),
            "lasso": {"A": A, "b": b, "lam": lam}}


def _sparse_positions(rng, rows: int, cols: int, count: int):
    """`count` distinct positions of a rows x cols matrix, uniform, in row-major order."""
    total = rows * cols
    count = min(int(count), total)
    if count * 4 >= total or (count * 100 >= total and total <= 1 << 31):
        idx = np.sort(rng.choice(total, size=count, replace=False))
    else:
        idx = np.unique(rng.integers(0, total, size=count))
        while idx.size < count:
            idx = np.unique(np.concatenate([idx, rng.integers(0, total, size=count - idx.size)]))
    return idx // cols, idx % cols


def lasso_paper(seed: int = 0, m: int = 70_000, n: int = 700_000, density: float = 1e-4):
    """The Lasso workload of the paper's experiments (Sec. 5.3; App. B.2):
    min ||A x - b||^2 + lam ||x||_1 with A (m x n) holding round(density m n) entries at
    uniform positions, each U[0, 1]; a ground truth x~ with N(0, 1) entries of which a random
    half is set to zero; b = A x~ + 1e-6 * 1; lam = ||A'b||_inf.  As the SOCP of App. B.2:
    variables w, r, y (m), x1, x2 (n each) with x = x1 - x2 >= 0 parts; zero rows w = 1 and
    y - A x1 + A x2 = -b; one second-order cone of dimension m + 2 holding
    ((w + r) / sqrt2, (w - r) / sqrt2, y), i.e. ||y||^2 <= 2 r when w = 1; objective
    2 r + lam 1'(x1 + x2).  The paper's sizes run from 1e4 x 1e5 (1e5 entries) to
    7.5e5 x 7.5e6 (5.6e8 entries)."""
    rng = np.random.default_rng(seed)
    m, n = int(m), int(n)
    ar, ac = _sparse_positions(rng, m, n, round(density * m * n))
    av = rng.random(ar.size)
    A = sp.csr_matrix((av, (ar, ac)), shape=(m, n))
    xt = rng.standard_normal(n)
    xt[rng.permutation(n)[: n // 2]] = 0.0
    b = A @ xt + 1e-6
    lam = float(np.abs(A.T @ b).max()) if A.nnz else 1.0
    nv = 2 + m + 2 * n
    iw, ir, iy, ix1, ix2 = 0, 1, 2, 2 + m, 2 + m + n
    s2 = np.sqrt(0.5)
    im = np.arange(m)
    rows = [np.zeros(1, np.int64), 1 + im, 1 + ar, 1 + ar, np.full(2, 1 + m), np.full(2, 2 + m), 3 + m + im]
    cols = [np.array([iw]), iy + im, ix1 + ac, ix2 + ac, np.array([iw, ir]), np.array([iw, ir]), iy + im]
    vals = [np.ones(1), np.ones(m), -av, av, np.array([s2, s2]), np.array([s2, -s2]), np.ones(m)]
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(2 * m + 3, nv))
    K.sort_indices()
    c = np.zeros(nv)
    c[ir] = 2.0
    c[ix1:] = lam
    h = np.zeros(2 * m + 3)
    h[0] = 1.0
    h[1:1 + m] = -b
    lb = np.full(nv, -np.inf)
    lb[ix1:] = 0.0
    ub = np.full(nv, np.inf)
    return {"name": "lasso_paper", "m": 2 * m + 3, "n": nv, "row_ptr": K.indptr.astype(np.int64),
            "col": K.indices.astype(np.int32), "val": K.data, "c": c, "h": h, "lb": lb, "ub": ub,
            "cone_types": np.asarray([ZERO, SOC], dtype=np.int32),
            "cone_dims": np.asarray([1 + m, m + 2], dtype=np.int64),
            "lasso": {"A": A, "b": b, "lam": lam}}


def lasso_paper_kp(seed: int = 0, m: int = 70_000, n: int = 700_000, density: float = 1e-4):
    """The same Lasso as lasso_paper (App. B.2), in the form the appendix writes it: the cone
    constraint on the variables themselves.  ((w + r)/sqrt2, (w - r)/sqrt2, y) in K_soc is
    (w, r, y) in K_rsoc (2 w r >= ||y||^2), a primal cone block x2 in K_p of m + 2 variables at
    the front; the rows are only the zero rows w = 1 and y - A x1 + A x2 = -b."""
    q = lasso_paper(seed, m, n, density)
    A, b = q["lasso"]["A"], q["lasso"]["b"]
    m, n = A.shape
    nv = 2 + m + 2 * n
    top = sp.csr_matrix((np.ones(1), (np.zeros(1, np.int64), np.zeros(1, np.int64))), shape=(1, nv))
    bot = sp.hstack([sp.csr_matrix((m, 2)), sp.identity(m, format="csr"), -A, A], format="csr")
    K = sp.vstack([top, bot], format="csr")
    K.sort_indices()
    h = np.concatenate([[1.0], -b])
    lb = q["lb"].copy()
    lb[:2] = -np.inf
    return {"name": "lasso_paper_kp", "m": 1 + m, "n": nv, "row_ptr": K.indptr.astype(np.int64),
            "col": K.indices.astype(np.int32), "val": K.data, "c": q["c"], "h": h, "lb": lb, "ub": q["ub"],
            "cone_types": np.asarray([ZERO], dtype=np.int32), "cone_dims": np.asarray([1 + m], dtype=np.int64),
            "pcone_types": np.asarray([RSOC], dtype=np.int32), "pcone_dims": np.asarray([m + 2], dtype=np.int64),
            "pcone_start": 0, "lasso": q["lasso"]}


def fisher_market(seed: int = 0, buyers: int = 100_000, goods: int = 1000, density: float = 0.2):
    """The Fisher market equilibrium workload of the paper's experiments (Sec. 5.2; App. B.1):
    max sum_i w_i log(sum_j U_ij X_ij) s.t. sum_i X_ij = b_j, X >= 0, with U (buyers x goods)
    holding round(density buyers goods) entries at uniform positions, each U[0, 1], budgets
    w_i ~ U[0, 1] and supplies b_j = 0.25.  As the exponential-cone program of App. B.1:
    min -w'p with t_i = sum_j U_ij X_ij and (p_i, 1, t_i) in K_exp (p_i <= log t_i).
    Variables X_ij only where U_ij > 0 (a buyer who does not value a good never receives it
    at equilibrium), then (p_i, t_i) per buyer; rows: goods clearing (zero), utility
    definitions (zero), then one exp cone per buyer.  The paper's sizes run from 1e2 x 5e3
    (1e5 entries) to 2.8e5 x 1e3 (5.5e7 entries)."""
    rng = np.random.default_rng(seed)
    mb, ng = int(buyers), int(goods)
    ur, uc = _sparse_positions(rng, mb, ng, round(density * mb * ng))
    uv = rng.random(ur.size)
    w = rng.random(mb)
    bsup = np.full(ng, 0.25)
    nx = ur.size
    n = nx + 2 * mb
    ip, it = nx, nx + mb
    ib = np.arange(mb)
    m = ng + mb + 3 * mb
    ex0 = ng + mb  # first exp row
    # K row by row, built directly in CSR: goods j (the X_ij of every buyer i that values j,
    # in buyer order), buyers i (their X_ij in good order, then -t_i), then per buyer the exp
    # rows p_i, (empty), t_i
    xid = np.arange(nx, dtype=np.int64)
    by_good = np.argsort(uc, kind="stable")
    cnt_g = np.bincount(uc, minlength=ng).astype(np.int64)
    cnt_b = np.bincount(ur, minlength=mb).astype(np.int64)
    lens = np.concatenate([cnt_g, cnt_b + 1, np.tile(np.array([1, 0, 1], np.int64), mb)])
    indptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(lens, out=indptr[1:])
    indices = np.empty(indptr[-1], dtype=np.int64)
    data = np.empty(indptr[-1])
    nb = int(indptr[ng])
    indices[:nb] = xid[by_good]
    data[:nb] = 1.0
    # buyer rows: entries of buyer i at indptr[ng + i] .. (cnt_b[i] X entries, then t_i)
    start = indptr[ng:ng + mb]
    pos_x = np.repeat(start, cnt_b) + (xid - np.repeat(np.cumsum(cnt_b) - cnt_b, cnt_b))
    indices[pos_x] = xid
    data[pos_x] = uv
    pos_t = start + cnt_b
    indices[pos_t] = it + ib
    data[pos_t] = -1.0
    e0 = indptr[ex0 + 3 * ib]
    indices[e0] = ip + ib
    data[e0] = 1.0
    e2 = indptr[ex0 + 3 * ib + 2]
    indices[e2] = it + ib
    data[e2] = 1.0
    K = sp.csr_matrix((data, indices.astype(np.int32), indptr), shape=(m, n))
    c = np.zeros(n)
    c[ip:ip + mb] = -w
    h = np.zeros(m)
    h[:ng] = bsup
    h[ex0 + 3 * ib + 1] = -1.0
    lb = np.full(n, -np.inf)
    lb[:nx] = 0.0
    ub = np.full(n, np.inf)
    types = np.concatenate([np.asarray([ZERO], dtype=np.int32), np.full(mb, EXP, dtype=np.int32)])
    dims = np.concatenate([np.asarray([ng + mb], dtype=np.int64), np.full(mb, 3, dtype=np.int64)])
    return {"name": "fisher_market", "m": m, "n": n, "row_ptr": K.indptr.astype(np.int64),
            "col": K.indices.astype(np.int32), "val": K.data, "c": c, "h": h, "lb": lb, "ub": ub,
            "cone_types": types, "cone_dims": dims,
            "fisher": {"U": sp.csr_matrix((uv, uc.astype(np.int32), np.concatenate([[0], np.cumsum(cnt_b)])),
                                          shape=(mb, ng)), "w": w, "b": bsup}}


def logistic_exp(seed: int = 2, n_samples: int = 200_000, n_features: int = 2000, density: float = 0.005,
                 lam_frac: float = 0.1):
    """l1-regularised logistic regression, min sum_i log(1 + exp(-b_i x_i'w)) + lam ||w||_1,
    as an exponential-cone program with two exp cones and one nonnegative row per sample
    (EXP = closure{(r, s, t): s > 0, t >= s exp(r / s)}).  Variables w+, w- >= 0 (w = w+ - w-,
    the l1 term through the bounds) and t, u, v free, one of each per sample:
        (-t_i, 1, u_i) in EXP                   i.e. u_i >= exp(-t_i),
        (-b_i x_i'w - t_i, 1, v_i) in EXP       i.e. v_i >= exp(-b_i x_i'w - t_i),
        1 - u_i - v_i >= 0,
    which together say t_i >= log(1 + exp(-b_i x_i'w)); objective 1't + lam 1'(w+ + w-).
    Rows: sample i's two cones at rows 6i .. 6i+5 (their s rows empty, h = -1), then the N
    nonnegative rows.  Variables: w+ (p), w- (p), t, u, v (N each).
    Data: each entry of X (N x p) present with probability `density`, N(0, 1) values; labels
    b_i = +-1 with probability 1/2; lam = lam_frac * ||X'b||_inf / 2 (w = 0 is optimal exactly
    when lam >= ||X'b||_inf / 2).  No known optimum: solutions are checked by the KKT evaluator
    and, on small instances, by a direct minimisation of the logistic objective."""
    rng = np.random.default_rng(seed)
    N, p = int(n_samples), int(n_features)
    deg = np.minimum(rng.binomial(p, density, N), p).astype(np.int64)
    xptr = np.zeros(N + 1, dtype=np.int64)
    np.cumsum(deg, out=xptr[1:])
    xcol = _unique_cols(rng, xptr, p)
    xval = rng.standard_normal(int(xptr[-1]))
    b = np.where(rng.random(N) < 0.5, 1.0, -1.0)
    X = sp.csr_matrix((xval, xcol, xptr), shape=(N, p))
    lam = lam_frac * 0.5 * float(np.abs(X.T @ b).max()) if N else 0.0
    n = 2 * p + 3 * N
    m = 7 * N
    it, iu, iv = 2 * p, 2 * p + N, 2 * p + 2 * N
    i = np.arange(N, dtype=np.int64)
    srow = np.repeat(i, deg)                       # sample of each entry of X
    bx = b[srow] * xval                            # b_i x_ij
    rows = [6 * i, 6 * i + 2, 6 * srow + 3, 6 * srow + 3, 6 * i + 3, 6 * i + 5, 6 * N + i, 6 * N + i]
    cols = [it + i, iu + i, xcol.astype(np.int64), p + xcol.astype(np.int64), it + i, iv + i, iu + i, iv + i]
    vals = [-np.ones(N), np.ones(N), -bx, bx, -np.ones(N), np.ones(N), -np.ones(N), -np.ones(N)]
    K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(m, n))
    K.sort_indices()
    c = np.zeros(n)
    c[:2 * p] = lam
    c[it:it + N] = 1.0
    h = np.zeros(m)
    h[6 * i + 1] = -1.0
    h[6 * i + 4] = -1.0
    h[6 * N:] = -1.0
    lb = np.full(n, -np.inf)
    lb[:2 * p] = 0.0
    ub = np.full(n, np.inf)
    types = np.concatenate([np.full(2 * N, EXP, dtype=np.int32), np.asarray([NONNEG] if N else [], dtype=np.int32)])
    dims = np.concatenate([np.full(2 * N, 3, dtype=np.int64), np.asarray([N] if N else [], dtype=np.int64)])
    return {"name": "logistic_exp", "m": m, "n": n, "row_ptr": K.indptr.astype(np.int64),
            "col": K.indices.astype(np.int32), "val": K.data, "c": c, "h": h, "lb": lb, "ub": ub,
            "cone_types": types, "cone_dims": dims,
            "logistic": {"X": X, "labels": b, "lam": lam}}


def lasso_batch(seed: int, count: int, n_lo: int = 50, n_hi: int = 1000):
    """`count` Lasso SOCPs of uneven sizes, n ~ U{n_lo..n_hi}, each from its own seed."""
    rng = np.random.default_rng(seed)
    sizes = rng.integers(n_lo, n_hi + 1, count)
    return [lasso_socp(int(seed) * 100_003 + k, int(nk)) for k, nk in enumerate(sizes)]


def portfolio_family(seed: int = 0, n_assets: int = 20_000, k: int = 100):
    """A parametric family of long-only factor-model portfolio SOCPs: F ~ N(0, 1/k) (n_assets x
    k, as N(0, 1/100) for k = 100), box [0, 0.05], budget 1'x = 1, factor exposures f = F'x and
    the risk bound ||f|| <= gamma as one SOC of dim k + 1; gamma is half the mean factor risk
    ||F'x_g|| of greedy box + budget portfolios x_g (the 1 / 0.05 best assets of five return
    draws).  Instances differ only in the expected returns mu ~ N(0.05, 0.02) per asset."""
    rng = np.random.default_rng(seed)
    F = rng.normal(0.0, 1.0 / np.sqrt(k), (n_assets, k))
    cap = 0.05
    top = int(round(1.0 / cap))
    risks = []
    for _ in range(5):
        mu = rng.normal(0.05, 0.02, n_assets)
        xg = np.zeros(n_assets)
        xg[np.argsort(-mu)[:top]] = cap
        risks.append(np.linalg.norm(F.T @ xg))
    return {"F": F, "gamma": 0.5 * float(np.mean(risks)), "cap": cap, "seed": seed}


def portfolio_mu(family, seed: int):
    """Expected returns of one instance of the family: N(0.05, 0.02) per asset."""
    return np.random.default_rng(10_000_019 + seed).normal(0.05, 0.02, family["F"].shape[0])


def portfolio_socp(family, mu):
    """min -mu'x s.t. 1'x = 1, f - F'x = 0 (zero rows), (gamma, f) in SOC(k + 1), 0 <= x <= cap,
    f free.  Variables (x, f); rows: budget, k exposure rows, then the SOC block whose first
    row is empty with h = -gamma."""
    F, gamma, cap = family["F"], family["gamma"], family["cap"]
    na, k = F.shape
    nv = na + k
    rows = [np.zeros(na, dtype=np.int64)]
    cols = [np.arange(na)]
    vals = [np.ones(na)]
    for j in range(k):
        rows.append(np.full(na + 1, 1 + j))
        cols.append(np.concatenate([np.arange(na), [na + j]]))
        vals.append(np.concatenate([-F[:, j], [1.0]]))
    o = 1 + k
    rows.append(o + 1 + np.arange(k))
    cols.append(na + np.arange(k))
    vals.append(np.ones(k))
    R = np.concatenate(rows)
    C = np.concatenate(cols)
    V = np.concatenate(vals)
    m = 2 * k + 2
    M = sp.csr_matrix((V, (R, C)), shape=(m, nv))
    M.sort_indices()
    c = np.concatenate([-np.asarray(mu, dtype=float), np.zeros(k)])
    h = np.zeros(m)
    h[0] = 1.0
    h[o] = -gamma
    lb = np.concatenate([np.zeros(na), np.full(k, -np.inf)])
    ub = np.concatenate([np.full(na, cap), np.full(k, np.inf)])
    return {"name": "portfolio_socp", "m": m, "n": nv, "row_ptr": M.indptr.astype(np.int64),
            "col": M.indices.astype(np.int32), "val": M.data, "c": c, "h": h, "lb": lb, "ub": ub,
            "cone_types": np.asarray([ZERO, SOC], dtype=np.int32),
            "cone_dims": np.asarray([1 + k, k + 1], dtype=np.int64)}


def portfolio_features(family, mu):
    """Summary of the returns fed to the warm-start network (k + 7 values): the factor
    exposures F'mu / n of the returns, and the mean, standard deviation, median, 90 % and
    99 % quantiles, maximum and top-(1/cap) mean of mu."""
    F, cap = family["F"], family["cap"]
    mu = np.asarray(mu, dtype=float)
    top = np.sort(mu)[::-1][:int(round(1.0 / cap))]
    q = np.quantile(mu, [0.5, 0.9, 0.99])
    stats = [mu.mean(), mu.std(), q[0], q[1], q[2], mu.max(), top.mean()]
    return np.concatenate([F.T @ mu / np.sqrt(F.shape[0]), stats]).astype(np.float32)
