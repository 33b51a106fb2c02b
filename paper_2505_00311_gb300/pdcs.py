"""ctypes binding of the C ABI in ``include/pdcs.h`` (argument marshalling only).

Every computation runs in the CUDA library ``_build/libpdcs.so``; there is no
fallback.  If the library has not been built, or no CUDA device is present,
the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdcs.so")

CONE_ZERO, CONE_NONNEG, CONE_SOC, CONE_RSOC, CONE_EXP, CONE_EXP_DUAL = 0, 1, 2, 3, 4, 5
SPMV_AUTO, SPMV_BINNED, SPMV_SLICED = 0, 1, 2
OK, ERR_INVALID, ERR_CUDA, ERR_OOM, ERR_NUMERIC, ERR_DEVICE_TIMEOUT, MAX_ITER, TIME_LIMIT = 0, 1, 2, 3, 4, 5, 10, 11
RESCALE_NONE, RESCALE_COORD, RESCALE_BLOCK = 0, 1, 2
STEP_ADAPTIVE, STEP_CONSTANT, STEP_PLAIN = 0, 1, 2
PRECISION_FP64, PRECISION_FP32 = 0, 1
STATUS_NAMES = {0: "ok", 1: "invalid", 2: "cuda", 3: "oom", 4: "numeric", 5: "device_timeout", 10: "max_iter",
                11: "time_limit"}

_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)
_fp = ctypes.POINTER(ctypes.c_float)


class pdcs_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", _i64p), ("col", _i32p), ("val", _dp)]


class pdcs_cone(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("dim", ctypes.c_int64)]


class pdcs_options(ctypes.Structure):
    _fields_ = [("rescale", ctypes.c_int32), ("ruiz_iters", ctypes.c_int32), ("pock_chambolle", ctypes.c_int32),
                ("step_mode", ctypes.c_int32), ("check_period", ctypes.c_int32), ("beta", ctypes.c_double),
                ("power_iters", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("fp32_switch_tol", ctypes.c_double), ("use_graphs", ctypes.c_int32),
                ("spmv_lanes", ctypes.c_int32), ("time_limit", ctypes.c_double),
                ("exp_mlp", ctypes.c_void_p), ("spmv_autotune", ctypes.c_int32), ("batch_blocks", ctypes.c_int32),
                ("spmv_format", ctypes.c_int32), ("soc_lane_entries", ctypes.c_int32),
                ("soc_grid_dim", ctypes.c_int32), ("fuse_primal", ctypes.c_int32),
                ("primal_cones", ctypes.c_void_p), ("n_primal_cones", ctypes.c_int64),
                ("primal_cone_start", ctypes.c_int64)]


class pdcs_info(ctypes.Structure):
    _fields_ = [("attempts", ctypes.c_int64), ("accepted", ctypes.c_int64), ("restarts", ctypes.c_int64),
                ("err_p", ctypes.c_double), ("err_d", ctypes.c_double), ("err_gap", ctypes.c_double),
                ("pobj", ctypes.c_double), ("dobj", ctypes.c_double), ("eta", ctypes.c_double),
                ("omega", ctypes.c_double), ("setup_seconds", ctypes.c_double),
                ("solve_seconds", ctypes.c_double), ("status", ctypes.c_int32), ("fp64_phase", ctypes.c_int32),
                ("kernel_launches", ctypes.c_int64), ("spmv_plan", ctypes.c_int32 * 4), ("spmv_format", ctypes.c_int32),
                ("soc_grid_cones", ctypes.c_int32), ("fuse_primal", ctypes.c_int32)]

    def as_dict(self):
        return {k: (list(getattr(self, k)) if isinstance(getattr(self, k), ctypes.Array) else getattr(self, k))
                for k, _ in self._fields_}


class pdcs_state(ctypes.Structure):
    _fields_ = [("eta", ctypes.c_double), ("omega", ctypes.c_double), ("wsum", ctypes.c_double),
                ("phi0", ctypes.c_double), ("phi_prev", ctypes.c_double), ("comp0", ctypes.c_double * 3),
                ("attempts", ctypes.c_int64), ("accepted", ctypes.c_int64), ("k", ctypes.c_int64),
                ("restarts", ctypes.c_int64), ("started", ctypes.c_int32), ("status", ctypes.c_int32)]


STATE_N = ["x", "xhat", "x0", "xsum", "kty", "kty0"]
STATE_M = ["y", "yhat", "y0", "ysum", "kx", "kx0"]


class pdcs_state_arrays(ctypes.Structure):
    _fields_ = [(k, _dp) for k in ["x", "xhat", "x0", "xsum", "y", "yhat", "y0", "ysum", "kx", "kx0", "kty", "kty0"]] + \
        [("soc_root", _fp), ("exp_root", _fp)]


_lock = threading.Lock()
_lib = None

# exported symbols and their signatures (kept in step with include/pdcs.h)
SIGNATURES = {
    "pdcs_default_options": (None, [ctypes.POINTER(pdcs_options)]),
    "pdcs_create": (ctypes.c_int, [ctypes.POINTER(pdcs_csr), _dp, _dp, _dp, _dp, ctypes.POINTER(pdcs_cone),
                                   ctypes.c_int64, ctypes.POINTER(pdcs_options), ctypes.c_void_p,
                                   ctypes.POINTER(ctypes.c_void_p)]),
    "pdcs_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.POINTER(pdcs_info)]),
    "pdcs_get_solution": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp]),
    "pdcs_get_iterate": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp]),
    "pdcs_get_scaling": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp]),
    "pdcs_get_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pdcs_info)]),
    "pdcs_set_warm_start": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, ctypes.c_double]),
    "pdcs_kernel_times": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64, _dp, _i64p]),
    "pdcs_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pdcs_state), ctypes.POINTER(pdcs_state_arrays)]),
    "pdcs_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(pdcs_state), ctypes.POINTER(pdcs_state_arrays)]),
    "pdcs_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "pdcs_destroy": (None, [ctypes.c_void_p]),
    "pdcs_proj_cones_device": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                              ctypes.POINTER(pdcs_cone), ctypes.c_int64, ctypes.c_int32,
                                              ctypes.c_void_p, ctypes.c_void_p]),
    "pdcs_proj_cones_device_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                      ctypes.POINTER(pdcs_cone), ctypes.c_int64, ctypes.c_int32,
                                                      ctypes.c_void_p, ctypes.c_void_p]),
    "pdcs_proj_plan_create": (ctypes.c_int, [ctypes.c_int64, ctypes.POINTER(pdcs_cone), ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "pdcs_proj_plan_run": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                          ctypes.c_void_p, ctypes.c_void_p]),
    "pdcs_proj_plan_check": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "pdcs_proj_plan_destroy": (None, [ctypes.c_void_p]),
    "pdcs_exp_mlp_dataset": (ctypes.c_int, [ctypes.c_int64, _dp, _dp, _fp, _fp, _i64p]),
    "pdcs_exp_mlp_loss_grad": (ctypes.c_int, [ctypes.c_int64, _fp, _fp, _fp, _fp, _fp]),
    "pdcs_exp_mlp_train": (ctypes.c_int, [ctypes.c_int64, _fp, _fp, ctypes.c_int32, ctypes.c_int32, ctypes.c_float,
                                          ctypes.c_uint64, _fp, _fp]),
    "pdcs_exp_proj_stats": (ctypes.c_int, [ctypes.c_int64, _dp, _dp, _fp, _dp, _i32p]),
    "pdcs_batch_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_void_p)]),
    "pdcs_batch_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, _i64p]),
    "pdcs_batch_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "pdcs_batch_destroy": (None, [ctypes.c_void_p]),
    "pdcs_mlp_params": (ctypes.c_int64, [ctypes.c_int32, _i32p]),
    "pdcs_mlp_forward": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.c_int64, _fp, _fp, _fp]),
    "pdcs_mlp_forward_bf16": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.c_int64, _fp, _fp, _fp]),
    "pdcs_mlp_loss_grad": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.c_int64, _fp, _fp, _fp, _fp, _fp]),
    "pdcs_mlp_train": (ctypes.c_int, [ctypes.c_int32, _i32p, ctypes.c_int64, _fp, _fp, ctypes.c_int32,
                                      ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _fp, _fp]),
}
EXP_MLP_IN, EXP_MLP_HIDDEN = 9, 32
EXP_MLP_PARAMS = EXP_MLP_HIDDEN * EXP_MLP_IN + EXP_MLP_HIDDEN + EXP_MLP_HIDDEN * EXP_MLP_HIDDEN + 2 * EXP_MLP_HIDDEN + 1
NOALLOC_MAX_CONES = 262144


def lib():
    """Loads the CUDA library (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("CUDA library %s is missing: run paper_2505_00311_gb300.build.build()" % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


class PdcsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (%d): %s" % (STATUS_NAMES.get(status, "?"), status, msg))
        self.status = status


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return None if a is None else a.ctypes.data_as(t)


def pdcs_default_options(**kw):
    o = pdcs_options()
    lib().pdcs_default_options(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _cones(types, dims):
    """The cone list as a pdcs_cone array (built in one numpy pass)."""
    types = np.asarray(types)
    dims = np.asarray(dims)
    rec = np.zeros(len(types), dtype=[("type", "<i4"), ("pad", "<i4"), ("dim", "<i8")])
    assert rec.itemsize == ctypes.sizeof(pdcs_cone)
    rec["type"] = types
    rec["dim"] = dims
    arr = (pdcs_cone * len(types)).from_buffer_copy(rec.tobytes())
    return arr


def pdcs_last_error(ctx=None):
    s = lib().pdcs_last_error(ctx)
    return s.decode() if s else ""


def pdcs_create(prob, options=None, stream=None):
    """Creates a solver for ``prob`` (dict with m, n, row_ptr, col, val, c, h, lb, ub,
    cone_types, cone_dims and optionally the primal cone blocks pcone_types, pcone_dims,
    pcone_start; host arrays).  Returns the opaque context handle."""
    rp = np.ascontiguousarray(prob["row_ptr"], dtype=np.int64)
    ci = np.ascontiguousarray(prob["col"], dtype=np.int32)
    val = _f64(prob["val"])
    c = _f64(prob["c"])
    h = _f64(prob["h"])
    lb = None if prob.get("lb") is None else _f64(prob["lb"])
    ub = None if prob.get("ub") is None else _f64(prob["ub"])
    K = pdcs_csr(int(prob["m"]), int(prob["n"]), int(rp[-1]), _ptr(rp, _i64p), _ptr(ci, _i32p), _ptr(val))
    cones = _cones(prob["cone_types"], prob["cone_dims"])
    opt = options if options is not None else pdcs_default_options()
    pcones = None
    if len(prob.get("pcone_types", [])):  # copied by pdcs_create
        pcones = _cones(prob["pcone_types"], prob["pcone_dims"])
        opt = pdcs_options.from_buffer_copy(opt)
        opt.primal_cones = ctypes.addressof(pcones)
        opt.n_primal_cones = len(pcones)
        opt.primal_cone_start = int(prob.get("pcone_start", 0))
    out = ctypes.c_void_p()
    st = lib().pdcs_create(ctypes.byref(K), _ptr(c), _ptr(h), _ptr(lb), _ptr(ub), cones, len(cones),
                           ctypes.byref(opt), stream, ctypes.byref(out))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(None))
    return out.value


def pdcs_solve(ctx, tol, max_iter):
    info = pdcs_info()
    st = lib().pdcs_solve(ctx, float(tol), int(max_iter), ctypes.byref(info))
    if st not in (OK, MAX_ITER, TIME_LIMIT):
        raise PdcsError(st, pdcs_last_error(ctx))
    return st, info.as_dict()


def pdcs_get_solution(ctx, m, n, want_lambda=False):
    x, y = np.empty(n), np.empty(m)
    lam = np.empty(n) if want_lambda else None
    st = lib().pdcs_get_solution(ctx, _ptr(x), _ptr(y), _ptr(lam))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))
    return (x, y, lam) if want_lambda else (x, y)


def pdcs_get_iterate(ctx, m, n):
    x, y, xh, yh = np.empty(n), np.empty(m), np.empty(n), np.empty(m)
    st = lib().pdcs_get_iterate(ctx, _ptr(x), _ptr(y), _ptr(xh), _ptr(yh))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))
    return x, y, xh, yh


def pdcs_get_scaling(ctx, m, n):
    dr, dc = np.empty(m), np.empty(n)
    st = lib().pdcs_get_scaling(ctx, _ptr(dr), _ptr(dc))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))
    return dr, dc


def pdcs_get_info(ctx):
    info = pdcs_info()
    st = lib().pdcs_get_info(ctx, ctypes.byref(info))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))
    return info.as_dict()


def pdcs_set_warm_start(ctx, x=None, y=None, omega=0.0):
    xa = None if x is None else _f64(x)
    ya = None if y is None else _f64(y)
    st = lib().pdcs_set_warm_start(ctx, _ptr(xa), _ptr(ya), float(omega))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))


def pdcs_get_state(ctx, m, n, n_soc=0, n_exp=0):
    """The iterate state in the rescaled program's coordinates: dict of the vectors
    (x, xhat, x0, xsum, kty, kty0: n; y, yhat, y0, ysum, kx, kx0: m), the root-search
    starting points (soc_root: n_soc, exp_root: n_exp) and the scalars."""
    vec = {k: np.empty(n) for k in STATE_N}
    vec.update({k: np.empty(m) for k in STATE_M})
    roots = {"soc_root": np.empty(max(n_soc, 1), np.float32), "exp_root": np.empty(max(n_exp, 1), np.float32)}
    arr = pdcs_state_arrays(**{k: _ptr(v) for k, v in vec.items()},
                            **{k: _ptr(v, _fp) for k, v in roots.items()})
    vec["soc_root"], vec["exp_root"] = roots["soc_root"][:n_soc], roots["exp_root"][:n_exp]
    st = pdcs_state()
    r = lib().pdcs_get_state(ctx, ctypes.byref(st), ctypes.byref(arr))
    if r != OK:
        raise PdcsError(r, pdcs_last_error(ctx))
    for f, _ in pdcs_state._fields_:
        v = getattr(st, f)
        vec[f] = list(v) if isinstance(v, ctypes.Array) else v
    return vec


def pdcs_set_state(ctx, state):
    """Restores a state (as returned by pdcs_get_state; the product vectors and the sums
    may be absent: recomputed / zero)."""
    keep = {k: _f64(state[k]) for k in STATE_N + STATE_M if state.get(k) is not None}
    roots = {k: np.ascontiguousarray(state[k], np.float32) for k in ("soc_root", "exp_root")
             if state.get(k) is not None and len(state[k])}
    arr = pdcs_state_arrays(**{k: _ptr(v) for k, v in keep.items()},
                            **{k: _ptr(v, _fp) for k, v in roots.items()})
    st = pdcs_state()
    for f, _ in pdcs_state._fields_:
        if f == "comp0":
            st.comp0[:] = [float(x) for x in state["comp0"]]
        elif f in ("eta", "omega", "wsum", "phi0", "phi_prev"):
            setattr(st, f, float(state[f]))
        else:
            setattr(st, f, int(state[f]))
    r = lib().pdcs_set_state(ctx, ctypes.byref(st), ctypes.byref(arr))
    if r != OK:
        raise PdcsError(r, pdcs_last_error(ctx))


KERNEL_CLASSES = ["primal_update", "spmv_K", "dual_update", "spmv_KT", "check", "check_flush", "check_cand_primal",
                  "check_cand_dual", "check_spmv", "check_kkt_primal", "check_kkt_dual", "check_restart"]


def pdcs_kernel_times(ctx, attempts):
    """Average ms per launch of each kernel class over `attempts` evaluations (CUDA events)."""
    ms = np.zeros(len(KERNEL_CLASSES))
    cnt = np.zeros(len(KERNEL_CLASSES), dtype=np.int64)
    st = lib().pdcs_kernel_times(ctx, int(attempts), _ptr(ms), _ptr(cnt, _i64p))
    if st != OK:
        raise PdcsError(st, pdcs_last_error(ctx))
    return dict(zip(KERNEL_CLASSES, ms.tolist())), dict(zip(KERNEL_CLASSES, cnt.tolist()))


def pdcs_destroy(ctx):
    if ctx:
        lib().pdcs_destroy(ctx)


def pdcs_proj_cones_device(v_ptr, d_ptr, m, types, dims, dual, out_ptr, stream=None):
    """Device-pointer projection (pointers are integers, e.g. torch ``data_ptr()``)."""
    cones = _cones(types, dims)
    st = lib().pdcs_proj_cones_device(v_ptr, d_ptr, int(m), cones, len(cones), int(dual), out_ptr, stream)
    if st != OK:
        raise PdcsError(st, "pdcs_proj_cones_device failed")


def pdcs_proj_cones_device_noalloc(v_ptr, d_ptr, m, types, dims, dual, out_ptr, stream=None):
    """As pdcs_proj_cones_device, without any device allocation (scratch in a fixed
    device array of NOALLOC_MAX_CONES cones); returns the pdcs_status code."""
    cones = _cones(types, dims)
    return lib().pdcs_proj_cones_device_noalloc(v_ptr, d_ptr, int(m), cones, len(cones), int(dual), out_ptr, stream)


class ProjPlan:
    """A projection plan (pdcs_proj_plan_*): the cone layout built once, then runs that
    only enqueue kernels.  Pointers are integers (e.g. torch ``data_ptr()``)."""

    def __init__(self, m, types, dims, stream=None):
        self._cones = _cones(types, dims)
        self.plan = ctypes.c_void_p()
        st = lib().pdcs_proj_plan_create(int(m), self._cones, len(self._cones), stream, ctypes.byref(self.plan))
        if st != OK:
            raise PdcsError(st, "pdcs_proj_plan_create failed")

    def run(self, v_ptr, d_ptr, dual, out_ptr, stream=None):
        st = lib().pdcs_proj_plan_run(self.plan, v_ptr, d_ptr, int(dual), out_ptr, stream)
        if st != OK:
            raise PdcsError(st, "pdcs_proj_plan_run failed")

    def check(self, stream=None):
        return lib().pdcs_proj_plan_check(self.plan, stream)

    def close(self):
        if self.plan:
            lib().pdcs_proj_plan_destroy(self.plan)
            self.plan = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owning wrapper of one solver context."""

    def __init__(self, prob, stream=None, **options):
        self.m, self.n = int(prob["m"]), int(prob["n"])
        kinds = np.asarray(prob["cone_types"])
        self.n_soc, self.n_exp = int(np.sum((kinds == CONE_SOC) | (kinds == CONE_RSOC))), int(np.sum((kinds == CONE_EXP) | (kinds == CONE_EXP_DUAL)))
        mlp = options.pop("exp_mlp", None)
        self.options = pdcs_default_options(**options)
        if mlp is not None:  # weights of the learned exp starting point, copied by pdcs_create
            mlp = np.ascontiguousarray(mlp, dtype=np.float32)
            if mlp.size != EXP_MLP_PARAMS:
                raise ValueError("exp_mlp needs %d weights" % EXP_MLP_PARAMS)
            self.options.exp_mlp = mlp.ctypes.data
        self.ctx = pdcs_create(prob, self.options, stream)

    def solve(self, tol=1e-6, max_iter=1_000_000):
        return pdcs_solve(self.ctx, tol, max_iter)

    def run(self, attempts):
        """Exactly ``attempts`` PDHG evaluations with termination off."""
        return pdcs_solve(self.ctx, 0.0, attempts)

    def solution(self, want_lambda=False):
        return pdcs_get_solution(self.ctx, self.m, self.n, want_lambda)

    def iterate(self):
        return pdcs_get_iterate(self.ctx, self.m, self.n)

    def scaling(self):
        return pdcs_get_scaling(self.ctx, self.m, self.n)

    def info(self):
        return pdcs_get_info(self.ctx)

    def kernel_times(self, attempts):
        return pdcs_kernel_times(self.ctx, attempts)

    def warm_start(self, x=None, y=None, omega=0.0):
        pdcs_set_warm_start(self.ctx, x, y, omega)

    def get_state(self):
        return pdcs_get_state(self.ctx, self.m, self.n, self.n_soc, self.n_exp)

    def set_state(self, state):
        pdcs_set_state(self.ctx, state)

    def close(self):
        if self.ctx:
            pdcs_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# learned starting point of the exponential-cone root search
# ---------------------------------------------------------------------------
def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _check(st):
    if st != OK:
        raise PdcsError(st, pdcs_last_error())


def exp_mlp_dataset(v, d):
    """Case-4 training pairs from the plain projector: (features k x 9, target L, k)."""
    v, d = _f64(v).reshape(-1, 3), _f64(d).reshape(-1, 3)
    n = v.shape[0]
    feats = np.empty((n, EXP_MLP_IN), dtype=np.float32)
    target = np.empty(n, dtype=np.float32)
    kept = ctypes.c_int64(0)
    _check(lib().pdcs_exp_mlp_dataset(n, _ptr(v), _ptr(d), _ptr(feats, _fp), _ptr(target, _fp), ctypes.byref(kept)))
    k = kept.value
    return feats[:k].copy(), target[:k].copy()


def exp_mlp_loss_grad(feats, target, weights):
    feats, target, weights = _f32(feats), _f32(target), _f32(weights)
    grad = np.empty(EXP_MLP_PARAMS, dtype=np.float32)
    loss = np.empty(1, dtype=np.float32)
    _check(lib().pdcs_exp_mlp_loss_grad(target.size, _ptr(feats, _fp), _ptr(target, _fp), _ptr(weights, _fp),
                                        _ptr(grad, _fp), _ptr(loss, _fp)))
    return float(loss[0]), grad


def exp_mlp_train(feats, target, weights, steps=2000, batch=4096, lr=1e-3, seed=0):
    """Adam training on the GPU; returns (trained weights, per-step minibatch loss)."""
    feats, target = _f32(feats), _f32(target)
    w = _f32(weights).copy()
    trace = np.empty(max(steps, 1), dtype=np.float32)
    _check(lib().pdcs_exp_mlp_train(target.size, _ptr(feats, _fp), _ptr(target, _fp), int(steps), int(batch),
                                    float(lr), int(seed), _ptr(w, _fp), _ptr(trace, _fp)))
    return w, trace[:steps]


def exp_proj_stats(v, d, weights=None):
    """Cold-start projections onto D K_exp: (out n x 3, evals n x 2: FP32, FP64 evaluations)."""
    v, d = _f64(v).reshape(-1, 3), _f64(d).reshape(-1, 3)
    n = v.shape[0]
    out = np.empty((n, 3))
    ev = np.empty((n, 2), dtype=np.int32)
    w = None if weights is None else _f32(weights)
    _check(lib().pdcs_exp_proj_stats(n, _ptr(v), _ptr(d), _ptr(w, _fp), _ptr(out), _ptr(ev, _i32p)))
    return out, ev


def exp_mlp_init(seed=0):
    """He-initialised weights (W1, b1, W2, b2, w3, b3), seeded."""
    rng = np.random.default_rng(seed)
    H, I = EXP_MLP_HIDDEN, EXP_MLP_IN
    parts = [rng.normal(0, np.sqrt(2.0 / I), H * I), np.zeros(H), rng.normal(0, np.sqrt(2.0 / H), H * H),
             np.zeros(H), rng.normal(0, np.sqrt(1.0 / H), H), np.zeros(1)]
    return np.concatenate(parts).astype(np.float32)


# ---------------------------------------------------------------------------
# batches of programs
# ---------------------------------------------------------------------------
class Batch:
    """Solves the programs of several Solver objects together (they must have been made
    with the same batch_blocks > 0 and not solved yet).  The solvers keep their
    solutions and info; close them after the batch."""

    def __init__(self, solvers):
        self.solvers = list(solvers)
        arr = (ctypes.c_void_p * len(self.solvers))(*[s.ctx for s in self.solvers])
        out = ctypes.c_void_p()
        st = lib().pdcs_batch_create(arr, len(self.solvers), ctypes.byref(out))
        if st != OK:
            raise PdcsError(st, lib().pdcs_batch_last_error(None).decode())
        self.b = out.value

    def solve(self, tol=1e-6, max_iter=1_000_000):
        n = ctypes.c_int64(0)
        st = lib().pdcs_batch_solve(self.b, float(tol), int(max_iter), ctypes.byref(n))
        if st not in (OK, MAX_ITER):
            raise PdcsError(st, lib().pdcs_batch_last_error(self.b).decode())
        return st, n.value

    def close(self):
        if self.b:
            lib().pdcs_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# warm-start network (fully connected, ReLU hidden layers, linear output, MSE)
# ---------------------------------------------------------------------------
def _sizes(sizes):
    return np.ascontiguousarray(sizes, dtype=np.int32)


def mlp_params(sizes):
    sz = _sizes(sizes)
    return int(lib().pdcs_mlp_params(sz.size - 1, _ptr(sz, _i32p)))


def mlp_init(sizes, seed=0):
    """He-initialised parameters (per layer W then b), seeded."""
    rng = np.random.default_rng(seed)
    parts = []
    for din, dout in zip(sizes[:-1], sizes[1:]):
        parts += [rng.normal(0.0, np.sqrt(2.0 / din), dout * din), np.zeros(dout)]
    return np.concatenate(parts).astype(np.float32)


def mlp_forward(sizes, X, W):
    sz, X, W = _sizes(sizes), _f32(X), _f32(W)
    Y = np.empty((X.shape[0], sz[-1]), dtype=np.float32)
    _check(lib().pdcs_mlp_forward(sz.size - 1, _ptr(sz, _i32p), X.shape[0], _ptr(X, _fp), _ptr(W, _fp), _ptr(Y, _fp)))
    return Y


def mlp_forward_bf16(sizes, X, W):
    """mlp_forward with the layers' products on the tensor cores (BF16 operands, FP32 sums)."""
    sz, X, W = _sizes(sizes), _f32(X), _f32(W)
    Y = np.empty((X.shape[0], sz[-1]), dtype=np.float32)
    _check(lib().pdcs_mlp_forward_bf16(sz.size - 1, _ptr(sz, _i32p), X.shape[0], _ptr(X, _fp), _ptr(W, _fp),
                                       _ptr(Y, _fp)))
    return Y


def mlp_loss_grad(sizes, X, T, W):
    sz, X, T, W = _sizes(sizes), _f32(X), _f32(T), _f32(W)
    g = np.empty(W.size, dtype=np.float32)
    loss = np.empty(1, dtype=np.float32)
    _check(lib().pdcs_mlp_loss_grad(sz.size - 1, _ptr(sz, _i32p), X.shape[0], _ptr(X, _fp), _ptr(T, _fp),
                                    _ptr(W, _fp), _ptr(g, _fp), _ptr(loss, _fp)))
    return float(loss[0]), g


def mlp_train(sizes, X, T, W, steps=2000, batch=256, lr=1e-3, seed=0):
    sz, X, T = _sizes(sizes), _f32(X), _f32(T)
    w = _f32(W).copy()
    trace = np.empty(max(steps, 1), dtype=np.float32)
    _check(lib().pdcs_mlp_train(sz.size - 1, _ptr(sz, _i32p), X.shape[0], _ptr(X, _fp), _ptr(T, _fp), int(steps),
                                int(batch), float(lr), int(seed), _ptr(w, _fp), _ptr(trace, _fp)))
    return w, trace[:steps]
