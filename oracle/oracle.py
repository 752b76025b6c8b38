"""ctypes wrapper around ``pdhcg_oracle.c`` (test infrastructure only).

Argument marshalling only: every step of the oracle's arithmetic is in the C
file.  ``build()`` compiles it with gcc into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pdhcg_oracle.c")
_HDR = os.path.join(_HERE, "pdhcg_oracle.h")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

STATUS_NAMES = {
    0: "UNSOLVED",
    1: "OPTIMAL",
    2: "PRIMAL_INFEASIBLE",
    3: "DUAL_INFEASIBLE",
    4: "ITERATION_LIMIT",
    5: "TIME_LIMIT",
    6: "NUMERICAL_ERROR",
}
INNER = {"auto": 0, "diag": 1, "cg": 2, "bb": 3}


class _Csr(C.Structure):
    _fields_ = [
        ("nrows", C.c_int32),
        ("ncols", C.c_int32),
        ("rowptr", C.POINTER(C.c_int64)),
        ("col", C.POINTER(C.c_int32)),
        ("val", C.POINTER(C.c_double)),
    ]


class OracleParams(C.Structure):
    _fields_ = [
        ("eps_tol", C.c_double),
        ("eps_inf", C.c_double),
        ("time_limit_s", C.c_double),
        ("max_iter", C.c_int64),
        ("theta", C.c_double),
        ("kp", C.c_double),
        ("ki", C.c_double),
        ("kd", C.c_double),
        ("gamma_inner", C.c_double),
        ("eps_inner_min", C.c_double),
        ("eps_inner_first", C.c_double),
        ("k_eval", C.c_int32),
        ("inner", C.c_int32),
        ("max_inner_iter", C.c_int32),
        ("ruiz_iters", C.c_int32),
        ("restart_sufficient", C.c_double),
        ("restart_necessary", C.c_double),
        ("restart_artificial", C.c_double),
        ("power_max_iter", C.c_int32),
        ("pad0", C.c_int32),
        ("power_tol", C.c_double),
        ("eta_override", C.c_double),
        ("omega0_override", C.c_double),
        ("omega_clamp", C.c_double),
    ]


class OracleResult(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("inner_method", C.c_int32),
        ("iterations", C.c_int64),
        ("inner_iterations", C.c_int64),
        ("restarts", C.c_int64),
        ("r_primal", C.c_double),
        ("r_dual", C.c_double),
        ("r_gap", C.c_double),
        ("primal_obj", C.c_double),
        ("dual_obj", C.c_double),
        ("eta", C.c_double),
        ("omega", C.c_double),
        ("norm_A", C.c_double),
        ("solve_seconds", C.c_double),
        ("power_iters", C.c_int32),
        ("pad0", C.c_int32),
    ]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_ if not name.startswith("pad")}
        d["status_name"] = STATUS_NAMES.get(self.status, "?")
        return d


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    global _lib
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
            os.makedirs(_OUT_DIR, exist_ok=True)
            tmp = _LIB_PATH + f".{os.getpid()}.tmp"
            subprocess.check_call(
                ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                 "-D_POSIX_C_SOURCE=199309L", "-o", tmp, _SRC, "-lm"]
            )
            os.replace(tmp, _LIB_PATH)
            _lib = None
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB_PATH)
        lib.oracle_default_params.argtypes = [C.POINTER(OracleParams)]
        lib.oracle_solve.restype = C.c_int
        lib.oracle_norm_estimate.restype = C.c_double
        lib.oracle_inner_solve.restype = C.c_int32
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a, ctype=C.c_double):
    return a.ctypes.data_as(C.POINTER(ctype))


class _CsrHold:
    """Keeps numpy buffers alive while C reads them."""

    def __init__(self, M, nrows, ncols):
        self.indptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(M.indices, dtype=np.int32)
        self.data = _f64(M.data)
        self.s = _Csr(nrows, ncols, _ptr(self.indptr, C.c_int64), _ptr(self.indices, C.c_int32),
                      _ptr(self.data))


def default_params(**kw) -> OracleParams:
    p = OracleParams()
    _load().oracle_default_params(C.byref(p))
    for k, v in kw.items():
        if k == "inner" and isinstance(v, str):
            v = INNER[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def solve(qp, params: OracleParams | None = None, x0=None, y0=None, eps_trace_len: int = 0):
    """Solve ``qp`` (fields n, m, Q (csr or None), A (csr), c, lc, uc, lv, uv).

    Returns (x, y, result_dict[, eps_trace]).
    """
    lib = _load()
    if params is None:
        params = default_params()
    n, m = int(qp.n), int(qp.m)
    Qh = _CsrHold(qp.Q, n, n) if qp.Q is not None else None
    Ah = _CsrHold(qp.A, m, n)
    c, lc, uc, lv, uv = (_f64(v) for v in (qp.c, qp.lc, qp.uc, qp.lv, qp.uv))
    x = np.zeros(n)
    y = np.zeros(max(m, 1))
    res = OracleResult()
    x0a = _f64(x0) if x0 is not None else None
    y0a = _f64(y0) if y0 is not None else None
    tr = np.zeros(max(eps_trace_len, 1))
    R = getattr(qp, "R", None)
    if R is not None:
        # structured Q = P + R^T R (qp.Q holds P)
        Rh = _CsrHold(R, R.shape[0], n)
        lib.oracle_solve_qr(
            C.c_int32(n), C.c_int32(m), C.byref(Qh.s) if Qh else None, C.byref(Rh.s), C.byref(Ah.s),
            _ptr(c), _ptr(lc), _ptr(uc), _ptr(lv), _ptr(uv), C.byref(params),
            _ptr(x0a) if x0a is not None else None, _ptr(y0a) if y0a is not None else None,
            _ptr(x), _ptr(y), C.byref(res))
        return (x, y[:m], res.as_dict())
    lib.oracle_solve(
        C.c_int32(n), C.c_int32(m),
        C.byref(Qh.s) if Qh else None, C.byref(Ah.s),
        _ptr(c), _ptr(lc), _ptr(uc), _ptr(lv), _ptr(uv),
        C.byref(params),
        _ptr(x0a) if x0a is not None else None,
        _ptr(y0a) if y0a is not None else None,
        _ptr(x), _ptr(y), C.byref(res),
        _ptr(tr) if eps_trace_len else None, C.c_int32(eps_trace_len),
    )
    out = (x, y[:m], res.as_dict())
    if eps_trace_len:
        out = out + (tr[: min(eps_trace_len, int(res.iterations))],)
    return out


def ruiz(qp, passes: int = 10):
    """Ruiz factors (D, E) of the problem; with a factor qp.R the objective is
    Q + R^T R and the diagonal of R^T R enters the column maxima."""
    lib = _load()
    n, m = int(qp.n), int(qp.m)
    Qh = _CsrHold(qp.Q, n, n) if qp.Q is not None else None
    Ah = _CsrHold(qp.A, m, n)
    D = np.zeros(n)
    E = np.zeros(max(m, 1))
    R = getattr(qp, "R", None)
    if R is not None:
        Rh = _CsrHold(R, R.shape[0], n)
        lib.oracle_ruiz_qr(C.c_int32(n), C.c_int32(m), C.byref(Qh.s) if Qh else None, C.byref(Rh.s),
                           C.byref(Ah.s), C.c_int32(passes), _ptr(D), _ptr(E))
    else:
        lib.oracle_ruiz(C.c_int32(n), C.c_int32(m), C.byref(Qh.s) if Qh else None, C.byref(Ah.s),
                        C.c_int32(passes), _ptr(D), _ptr(E))
    return D, E[:m]


def norm_estimate(A, max_iter: int = 1000, tol: float = 1e-8):
    lib = _load()
    Ah = _CsrHold(A, A.shape[0], A.shape[1])
    it = C.c_int32(0)
    v = lib.oracle_norm_estimate(C.byref(Ah.s), Ah.s.val, C.c_int32(max_iter), C.c_double(tol),
                                 C.byref(it))
    return float(v), int(it.value)


def inner_solve(Q, lv, lu, tau, b, x0, eps, max_it, method):
    """One primal subproblem solve min_{l<=x<=u} 1/2 x^T (Q + I/tau) x - b^T x."""
    lib = _load()
    n = len(b)
    Qh = _CsrHold(Q, n, n) if Q is not None else None
    x = _f64(np.array(x0, dtype=np.float64, copy=True))
    lv, lu, b = _f64(lv), _f64(lu), _f64(b)
    steps = lib.oracle_inner_solve(C.c_int32(n), C.byref(Qh.s) if Qh else None, _ptr(lv), _ptr(lu),
                                   C.c_double(tau), _ptr(b), C.c_double(eps), C.c_int32(max_it),
                                   C.c_int32(INNER[method] if isinstance(method, str) else method),
                                   _ptr(x))
    return x, int(steps)


def kkt(n, m, x, y, Ax, ATy, Qx, c, lc, uc, lv, uv):
    """(r_primal, r_dual, r_gap, primal_obj, dual_obj) from unscaled products."""
    lib = _load()
    arrs = [_f64(v) for v in (x, y if m else np.zeros(1), Ax if m else np.zeros(1), ATy, Qx, c,
                              lc if m else np.zeros(1), uc if m else np.zeros(1), lv, uv)]
    out = np.zeros(6)
    lib.oracle_kkt(C.c_int32(n), C.c_int32(m), *[_ptr(a) for a in arrs], _ptr(out))
    return tuple(out[:5])


def pid_update(log_omega, e_sum, e_prev, dx, dy, kp=0.99, ki=0.01, kd=0.0, log_omega0=0.0,
               clamp=1e5):
    lib = _load()
    lw, es, ep = C.c_double(log_omega), C.c_double(e_sum), C.c_double(e_prev)
    lib.oracle_pid_update(C.byref(lw), C.byref(es), C.byref(ep), C.c_double(dx), C.c_double(dy),
                          C.c_double(kp), C.c_double(ki), C.c_double(kd), C.c_double(log_omega0),
                          C.c_double(clamp))
    return lw.value, es.value, ep.value
