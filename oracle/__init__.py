"""FP64 CPU oracle for the PDCS restarted-PDHG conic solver.

TEST INFRASTRUCTURE ONLY.  This package is the slow, plain reference that the
CUDA library is checked against.  Only the test suite, the smoke check and the
benchmark's CPU-baseline leg may import it; the product path never does.  It
shares no code with the CUDA library: the C sources in this folder are plain
single-threaded loops compiled with gcc, wrapped here with ctypes.

What each C function follows in the paper is documented in ``pdcs_oracle.h``,
``cones.c`` and ``solver.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liborc.so")
_SOURCES = ["cones.c", "solver.c"]
_lock = threading.Lock()
_lib = None

ZERO, NONNEG, SOC, RSOC, EXP, EXP_DUAL = 0, 1, 2, 3, 4, 5
RESCALE_NONE, RESCALE_COORD, RESCALE_BLOCK = 0, 1, 2
STEP_ADAPTIVE, STEP_CONSTANT, STEP_PLAIN = 0, 1, 2
RUNNING, CONVERGED, MAX_ITER = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle into ``_build/liborc.so`` with gcc (no -march flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    hdr = os.path.join(_HERE, "pdcs_oracle.h")
    newest = max(os.path.getmtime(p) for p in srcs + [hdr])
    if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= newest:
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c99", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", "-ffp-contract=off",
           "-o", tmp] + srcs + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Options(ctypes.Structure):
    _fields_ = [("rescale", ctypes.c_int), ("ruiz_iters", ctypes.c_int), ("pock_chambolle", ctypes.c_int),
                ("step_mode", ctypes.c_int), ("check_period", ctypes.c_int), ("beta", ctypes.c_double),
                ("power_iters", ctypes.c_int), ("pc_types", ctypes.POINTER(ctypes.c_int32)),
                ("pc_dims", ctypes.POINTER(ctypes.c_int64)), ("n_pc", ctypes.c_int64), ("pc_start", ctypes.c_int64)]


class _Kkt(ctypes.Structure):
    _fields_ = [("err_p", ctypes.c_double), ("err_d", ctypes.c_double), ("err_gap", ctypes.c_double),
                ("pobj", ctypes.c_double), ("dobj", ctypes.c_double)]


_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)
_i32p = ctypes.POINTER(ctypes.c_int32)


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_default_options.argtypes = [ctypes.POINTER(_Options)]
            L.orc_proj_soc.argtypes = [ctypes.c_double, _dp, _dp, ctypes.c_int64, _dp, _dp]
            L.orc_proj_rsoc.argtypes = [_dp, _dp, ctypes.c_int64, _dp]
            L.orc_proj_exp.argtypes = [_dp, _dp, _dp]
            L.orc_proj_exp_dual.argtypes = [_dp, _dp, _dp]
            L.orc_proj_cones.argtypes = [_dp, _dp, ctypes.c_int64, _i32p, _i64p, ctypes.c_int64, ctypes.c_int, _dp]
            L.orc_kkt_eval.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i32p, _dp, _dp, _dp, _dp, _dp,
                                       _i32p, _i64p, ctypes.c_int64, _dp, _dp, ctypes.POINTER(_Kkt)]
            L.orc_kkt_eval.restype = ctypes.c_int
            L.orc_kkt_eval_pc.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i32p, _dp, _dp, _dp, _dp, _dp,
                                          _i32p, _i64p, ctypes.c_int64, _i32p, _i64p, ctypes.c_int64,
                                          ctypes.c_int64, _dp, _dp, ctypes.POINTER(_Kkt)]
            L.orc_kkt_eval_pc.restype = ctypes.c_int
            L.orc_create.argtypes = [ctypes.c_int64, ctypes.c_int64, _i64p, _i32p, _dp, _dp, _dp, _dp, _dp,
                                     _i32p, _i64p, ctypes.c_int64, ctypes.POINTER(_Options)]
            L.orc_create.restype = ctypes.c_void_p
            L.orc_destroy.argtypes = [ctypes.c_void_p]
            L.orc_set_start.argtypes = [ctypes.c_void_p, _dp, _dp, ctypes.c_double]
            L.orc_run.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_int64]
            L.orc_run.restype = ctypes.c_int
            L.orc_get_scaling.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_get_iterate.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
            L.orc_get_solution.argtypes = [ctypes.c_void_p, _dp, _dp]
            L.orc_get_scalars.argtypes = [ctypes.c_void_p, _dp]
            L.orc_get_state.argtypes = [ctypes.c_void_p] + [_dp] * 9
            L.orc_set_state.argtypes = [ctypes.c_void_p] + [_dp] * 9
            L.orc_norm2_estimate.argtypes = [ctypes.c_void_p]
            L.orc_norm2_estimate.restype = ctypes.c_double
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


# ---- projections ---------------------------------------------------------
def proj_soc(v, d=None):
    """Projection of v = (t, x) onto D K_soc (Theorem 1)."""
    v = _f64(v)
    n = v.size - 1
    d = np.ones(v.size) if d is None else _f64(d)
    out = np.empty_like(v)
    ot = ctypes.c_double()
    xs = _f64(v[1:])
    ox = np.empty(n)
    lib().orc_proj_soc(float(v[0]), _ptr(xs), _ptr(d), n, ctypes.byref(ot), _ptr(ox))
    out[0] = ot.value
    out[1:] = ox
    return out


def proj_rsoc(v, d=None):
    v = _f64(v)
    d = np.ones(v.size) if d is None else _f64(d)
    out = np.empty_like(v)
    lib().orc_proj_rsoc(_ptr(v), _ptr(d), v.size, _ptr(out))
    return out


def proj_exp(v, d=None):
    """Projection of v = (r, s, t) onto D K_exp (Theorem 3)."""
    v = _f64(v)
    d = np.ones(3) if d is None else _f64(d)
    out = np.empty(3)
    lib().orc_proj_exp(_ptr(v), _ptr(d), _ptr(out))
    return out


def proj_exp_dual(v, d=None):
    v = _f64(v)
    d = np.ones(3) if d is None else _f64(d)
    out = np.empty(3)
    lib().orc_proj_exp_dual(_ptr(v), _ptr(d), _ptr(out))
    return out


def proj_cones(v, types, dims, d=None, dual=False):
    """Blockwise projection onto D C (dual=False) or D^{-1} C^* (dual=True)."""
    v = _f64(v)
    d = np.ones(v.size) if d is None else _f64(d)
    t = np.ascontiguousarray(types, dtype=np.int32)
    k = np.ascontiguousarray(dims, dtype=np.int64)
    out = np.empty_like(v)
    lib().orc_proj_cones(_ptr(v), _ptr(d), v.size, _ptr(t, _i32p), _ptr(k, _i64p), t.size, int(dual), _ptr(out))
    return out


# ---- problem handling ------------------------------------------------------
def _problem_arrays(prob):
    rp = np.ascontiguousarray(prob["row_ptr"], dtype=np.int64)
    ci = np.ascontiguousarray(prob["col"], dtype=np.int32)
    val = _f64(prob["val"])
    c = _f64(prob["c"])
    h = _f64(prob["h"])
    lb = None if prob.get("lb") is None else _f64(prob["lb"])
    ub = None if prob.get("ub") is None else _f64(prob["ub"])
    types = np.ascontiguousarray(prob["cone_types"], dtype=np.int32)
    dims = np.ascontiguousarray(prob["cone_dims"], dtype=np.int64)
    return rp, ci, val, c, h, lb, ub, types, dims


def _pc_arrays(prob):
    """Primal cone blocks of a problem dict (keys pcone_types, pcone_dims, pcone_start; absent:
    none): types (int32), sizes (int64), first variable."""
    t = np.ascontiguousarray(prob.get("pcone_types", []), dtype=np.int32)
    d = np.ascontiguousarray(prob.get("pcone_dims", []), dtype=np.int64)
    return t, d, int(prob.get("pcone_start", 0))


def kkt(prob, x, y):
    """Relative KKT errors (eq. PDCS_terminate_tolerance) of (x, y) for the original program."""
    rp, ci, val, c, h, lb, ub, types, dims = _problem_arrays(prob)
    pt, pd, ps = _pc_arrays(prob)
    x = _f64(x)
    y = _f64(y)
    out = _Kkt()
    rc = lib().orc_kkt_eval_pc(prob["m"], prob["n"], _ptr(rp, _i64p), _ptr(ci, _i32p), _ptr(val), _ptr(c),
                               _ptr(h), _ptr(lb), _ptr(ub), _ptr(types, _i32p), _ptr(dims, _i64p), types.size,
                               _ptr(pt if pt.size else None, _i32p), _ptr(pd if pd.size else None, _i64p),
                               pt.size, ps, _ptr(x), _ptr(y), ctypes.byref(out))
    if rc != 0:
        raise ValueError("invalid problem")
    return {"err_p": out.err_p, "err_d": out.err_d, "err_gap": out.err_gap, "pobj": out.pobj, "dobj": out.dobj}


def default_options(**kw):
    o = _Options()
    lib().orc_default_options(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Solver:
    """Restarted PDHG (Algorithm 1) on the CPU, step by step."""

    def __init__(self, prob, **opts):
        self._arrs = _problem_arrays(prob)
        rp, ci, val, c, h, lb, ub, types, dims = self._arrs
        self.m, self.n = int(prob["m"]), int(prob["n"])
        self._opt = default_options(**opts)
        self._pc = _pc_arrays(prob)
        if self._pc[0].size:
            self._opt.pc_types = self._pc[0].ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            self._opt.pc_dims = self._pc[1].ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
            self._opt.n_pc = self._pc[0].size
            self._opt.pc_start = self._pc[2]
        self._h = lib().orc_create(self.m, self.n, _ptr(rp, _i64p), _ptr(ci, _i32p), _ptr(val), _ptr(c), _ptr(h),
                                   _ptr(lb), _ptr(ub), _ptr(types, _i32p), _ptr(dims, _i64p), types.size,
                                   ctypes.byref(self._opt))
        if not self._h:
            raise ValueError("invalid problem")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().orc_destroy(h)
            self._h = None

    def set_start(self, x=None, y=None, omega=0.0):
        xa = None if x is None else _f64(x)
        ya = None if y is None else _f64(y)
        lib().orc_set_start(self._h, _ptr(xa), _ptr(ya), float(omega))

    def run(self, attempts, tol=0.0):
        return lib().orc_run(self._h, float(tol), int(attempts))

    def scaling(self):
        dr = np.empty(self.m)
        dc = np.empty(self.n)
        lib().orc_get_scaling(self._h, _ptr(dr), _ptr(dc))
        return dr, dc

    def iterate(self):
        x, y, xh, yh = np.empty(self.n), np.empty(self.m), np.empty(self.n), np.empty(self.m)
        lib().orc_get_iterate(self._h, _ptr(x), _ptr(y), _ptr(xh), _ptr(yh))
        return x, y, xh, yh

    def solution(self):
        x, y = np.empty(self.n), np.empty(self.m)
        lib().orc_get_solution(self._h, _ptr(x), _ptr(y))
        return x, y

    def scalars(self):
        o = np.empty(12)
        lib().orc_get_scalars(self._h, _ptr(o))
        keys = ["eta", "omega", "attempts", "accepted", "restarts", "inner_k", "status",
                "err_p", "err_d", "err_gap", "wsum", "phi0"]
        return dict(zip(keys, o.tolist()))

    def norm2(self):
        return lib().orc_norm2_estimate(self._h)

    STATE_VECTORS = ["x", "xh", "x0", "xsum", "y", "yh", "y0", "ysum"]
    STATE_SCALARS = ["eta", "omega", "wsum", "attempts", "accepted", "k", "restarts", "phi0", "phi_prev",
                     "comp0_rp2", "comp0_rd2", "comp0_gap", "status", "started"]

    def state(self):
        """Full iterate state in scaled coordinates (dict of arrays and scalars)."""
        vec = {k: np.empty(self.n if k.startswith("x") else self.m) for k in self.STATE_VECTORS}
        sc = np.empty(len(self.STATE_SCALARS))
        lib().orc_get_state(self._h, *[_ptr(vec[k]) for k in self.STATE_VECTORS], _ptr(sc))
        vec.update(dict(zip(self.STATE_SCALARS, sc.tolist())))
        return vec

    def set_state(self, st):
        """Restores a state returned by state() (arrays may be missing: left unchanged)."""
        vec = [None if st.get(k) is None else _f64(st[k]) for k in self.STATE_VECTORS]
        cur = self.state()
        sc = _f64([float(st.get(k, cur[k])) for k in self.STATE_SCALARS])
        lib().orc_set_state(self._h, *[_ptr(a) for a in vec], _ptr(sc))
