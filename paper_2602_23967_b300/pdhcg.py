"""Thin ctypes binding of libpdhcg.so (include/pdhcg.h).

Argument marshalling only: every step of the method runs in the library's CUDA
kernels.  Importing this module loads the in-tree ``libpdhcg.so``; if it is
missing the import fails loudly (there is no CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpdhcg.so")

OK, PENDING = 0, 1
E_INVALID, E_OOM, E_CUDA, E_BUSY, E_NOT_FOUND, E_DEVICE_TIMEOUT = -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "UNSOLVED", 1: "OPTIMAL", 2: "PRIMAL_INFEASIBLE", 3: "DUAL_INFEASIBLE",
                4: "ITERATION_LIMIT", 5: "TIME_LIMIT", 6: "NUMERICAL_ERROR"}
PRECISION = {"fp64": 0, "fp32": 1, "mixed": 2, "dfloat": 3}
INNER = {"auto": 0, "diag": 1, "cg": 2, "bb": 3, "cg_lifted": 4}


class PdhcgError(RuntimeError):
    def __init__(self, code, where, detail):
        super().__init__(f"{where}: {code} ({detail})")
        self.code = code


class Csr(C.Structure):
    # pdhcg_csr: the three pointers (const int64_t*, const int32_t*, const
    # double*) are filled with the arrays' integer addresses, which is much
    # cheaper than building typed ctypes pointers for thousands of problems
    _fields_ = [("nrows", C.c_int32), ("ncols", C.c_int32), ("nnz", C.c_int64),
                ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p)]


class Params(C.Structure):
    _fields_ = [
        ("struct_size", C.c_uint32), ("precision", C.c_int32),
        ("eps_tol", C.c_double), ("eps_inf", C.c_double), ("time_limit_s", C.c_double),
        ("max_iter", C.c_int64),
        ("theta", C.c_double), ("kp", C.c_double), ("ki", C.c_double), ("kd", C.c_double),
        ("gamma_inner", C.c_double), ("eps_inner_min", C.c_double), ("eps_inner_first", C.c_double),
        ("k_eval", C.c_int32), ("inner", C.c_int32), ("max_inner_iter", C.c_int32),
        ("ruiz_iters", C.c_int32),
        ("restart_sufficient", C.c_double), ("restart_necessary", C.c_double),
        ("restart_artificial", C.c_double),
        ("power_max_iter", C.c_int32), ("lanes_override", C.c_int32),
        ("power_tol", C.c_double), ("eta_override", C.c_double), ("omega0_override", C.c_double),
        ("omega_clamp", C.c_double),
        ("group_blocks", C.c_int32), ("device_timeout_ms", C.c_int32),
        ("sell_sigma", C.c_int32), ("long_row", C.c_int32), ("huge_row", C.c_int32),
        ("pool_ctas_per_sm", C.c_int32), ("pipeline", C.c_int32), ("pool_threads", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("inner_method", C.c_int32),
        ("iterations", C.c_int64), ("inner_iterations", C.c_int64), ("restarts", C.c_int64),
        ("r_primal", C.c_double), ("r_dual", C.c_double), ("r_gap", C.c_double),
        ("primal_obj", C.c_double), ("dual_obj", C.c_double),
        ("eta", C.c_double), ("omega", C.c_double), ("norm_A", C.c_double),
        ("solve_seconds", C.c_double), ("power_iters", C.c_int32), ("precision", C.c_int32),
        ("latency_seconds", C.c_double), ("form", C.c_int32), ("reserved", C.c_int32),
    ]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["status_name"] = STATUS_NAMES.get(self.status, "?")
        return d


class ProblemData(C.Structure):
    _fields_ = [("Q", C.POINTER(Csr)), ("A", C.POINTER(Csr)), ("c", C.POINTER(C.c_double)),
                ("lc", C.POINTER(C.c_double)), ("uc", C.POINTER(C.c_double)),
                ("lv", C.POINTER(C.c_double)), ("uv", C.POINTER(C.c_double))]


class Tuning(C.Structure):
    _fields_ = [("sell_sigma", C.c_int32), ("long_row", C.c_int32), ("huge_row", C.c_int32),
                ("group_blocks", C.c_int32), ("pool_ctas_per_sm", C.c_int32), ("pipeline", C.c_int32),
                ("candidates", C.c_int32),
                ("from_cache", C.c_int32), ("seconds_per_step", C.c_double),
                ("default_seconds_per_step", C.c_double), ("pool_threads", C.c_int32),
                ("reserved", C.c_int32)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("rejected", C.c_uint64), ("launches", C.c_uint64), ("live", C.c_int32),
                ("queued", C.c_int32), ("hbm_in_use", C.c_size_t), ("admit_seconds", C.c_double),
                ("slice_seconds", C.c_double), ("retire_seconds", C.c_double)]


_lib = None
_P = C.c_void_p
_D = C.POINTER(C.c_double)


def lib():
    """Load libpdhcg.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -m paper_2602_23967_b300.build`")
        L = C.CDLL(LIB_PATH)
        L.pdhcg_default_params.argtypes = [C.POINTER(Params)]
        L.pdhcg_create.argtypes = [C.POINTER(Csr), C.POINTER(Csr), _D, _D, _D, _D, _D,
                                   C.POINTER(Params), _P, C.POINTER(_P)]
        L.pdhcg_create_batch.argtypes = [C.c_int, C.POINTER(ProblemData), C.POINTER(Params), _P,
                                         C.POINTER(_P)]
        L.pdhcg_create_qr.argtypes = [C.POINTER(Csr), C.POINTER(Csr), C.POINTER(Csr), _D, _D, _D, _D, _D,
                                      C.POINTER(Params), _P, C.POINTER(_P)]
        L.pdhcg_solve.argtypes = [_P, _D, _D, C.POINTER(Result), _D, _D]
        L.pdhcg_solve_dev.argtypes = [_P, _P, _P, C.POINTER(Result), _P, _P]
        L.pdhcg_solve_batch.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(Result), C.POINTER(_D),
                                        C.POINTER(_D)]
        L.pdhcg_solve_batch_noalloc.argtypes = [C.POINTER(_P), C.c_int, C.POINTER(Result),
                                                C.POINTER(_P), C.POINTER(_P)]
        L.pdhcg_get_eta.argtypes = [_P, _D, _D]
        L.pdhcg_get_scaling.argtypes = [_P, _D, _D]
        L.pdhcg_get_info.argtypes = [_P, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                     C.POINTER(C.c_size_t)]
        L.pdhcg_get_phase_times.argtypes = [_P, _D]
        L.pdhcg_get_device.argtypes = [_P, C.POINTER(C.c_int32)]
        L.pdhcg_autotune.argtypes = [C.c_int, C.POINTER(ProblemData), C.POINTER(Params), _P, C.POINTER(Tuning)]
        L.pdhcg_destroy.argtypes = [_P]
        L.pdhcg_destroy.restype = None
        L.pdhcg_strerror.restype = C.c_char_p
        L.pdhcg_last_error.restype = C.c_char_p
        if hasattr(L, "pdhcg_server_create"):
            L.pdhcg_server_create.argtypes = [C.c_size_t, C.c_int, C.POINTER(Params), _P,
                                              C.POINTER(_P)]
            L.pdhcg_submit.argtypes = [_P, C.POINTER(Csr), C.POINTER(Csr), _D, _D, _D, _D, _D,
                                       C.POINTER(C.c_uint64)]
            L.pdhcg_poll.argtypes = [_P, C.c_uint64, C.POINTER(Result), _D, _D]
            L.pdhcg_server_get_stats.argtypes = [_P, C.POINTER(ServerStats)]
            L.pdhcg_server_destroy.argtypes = [_P]
            L.pdhcg_server_destroy.restype = None
        _lib = L
    return _lib


def check(code, where):
    if code < 0:
        L = lib()
        raise PdhcgError(code, where, (L.pdhcg_strerror(code) or b"").decode() + ": " +
                         (L.pdhcg_last_error() or b"").decode())
    return code


def default_params(**kw) -> Params:
    p = Params()
    check(lib().pdhcg_default_params(C.byref(p)), "pdhcg_default_params")
    for k, v in kw.items():
        if k == "precision" and isinstance(v, str):
            v = PRECISION[v]
        if k == "inner" and isinstance(v, str):
            v = INNER[v]
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _dp(a):
    return None if a is None else a.ctypes.data_as(_D)


class _CsrHold:
    def __init__(self, M, nrows, ncols):
        self.indptr = np.ascontiguousarray(M.indptr, dtype=np.int64)
        self.indices = np.ascontiguousarray(M.indices, dtype=np.int32)
        self.data = _f64(M.data)
        self.s = Csr(nrows, ncols, int(self.indptr[-1]) if len(self.indptr) else 0,
                     self.indptr.ctypes.data, self.indices.ctypes.data, self.data.ctypes.data)


def _qp_args(qp):
    n, m = int(qp.n), int(qp.m)
    hold = {"A": _CsrHold(qp.A, m, n)}
    if qp.Q is not None:
        hold["Q"] = _CsrHold(qp.Q, n, n)
    for k in ("c", "lc", "uc", "lv", "uv"):
        hold[k] = _f64(getattr(qp, k))
    return hold


class Problem:
    """A QP resident on the device (pdhcg_create)."""

    def __init__(self, qp, params: Params | None = None, stream=None, _handle=None):
        L = lib()
        self.n, self.m = int(qp.n), int(qp.m)
        self.params = params if params is not None else default_params()
        if _handle is not None:
            self.handle = _handle
            return
        h = _qp_args(qp)
        handle = _P()
        R = getattr(qp, "R", None)
        if R is not None:
            # structured objective Q + R^T R (pdhcg_create_qr)
            Rh = _CsrHold(R, int(R.shape[0]), self.n)
            rc = L.pdhcg_create_qr(C.byref(h["Q"].s) if "Q" in h else None, C.byref(Rh.s), C.byref(h["A"].s),
                                   _dp(h["c"]), _dp(h["lc"]), _dp(h["uc"]), _dp(h["lv"]), _dp(h["uv"]),
                                   C.byref(self.params), _P(stream) if stream else None, C.byref(handle))
            check(rc, "pdhcg_create_qr")
        else:
            rc = L.pdhcg_create(C.byref(h["Q"].s) if "Q" in h else None, C.byref(h["A"].s),
                                _dp(h["c"]), _dp(h["lc"]), _dp(h["uc"]), _dp(h["lv"]), _dp(h["uv"]),
                                C.byref(self.params), _P(stream) if stream else None, C.byref(handle))
            check(rc, "pdhcg_create")
        self.handle = handle

    def solve(self, x0=None, y0=None):
        x = np.zeros(self.n)
        y = np.zeros(max(self.m, 1))
        res = Result()
        x0 = _f64(x0) if x0 is not None else None
        y0 = _f64(y0) if y0 is not None else None
        check(lib().pdhcg_solve(self.handle, _dp(x0), _dp(y0), C.byref(res), _dp(x), _dp(y)),
              "pdhcg_solve")
        return x, y[: self.m], res.as_dict()

    def solve_dev(self, x_out, y_out, x0=None, y0=None):
        """Device-buffer solve: x_out / y_out (and optional x0 / y0) are float64 CUDA tensors."""
        res = Result()
        ptr = (lambda t: _P(t.data_ptr()) if t is not None else None)
        check(lib().pdhcg_solve_dev(self.handle, ptr(x0), ptr(y0), C.byref(res), ptr(x_out),
                                    ptr(y_out)), "pdhcg_solve_dev")
        return res.as_dict()

    def eta(self):
        e, a = C.c_double(), C.c_double()
        check(lib().pdhcg_get_eta(self.handle, C.byref(e), C.byref(a)), "pdhcg_get_eta")
        return e.value, a.value

    def scaling(self):
        D = np.zeros(self.n)
        E = np.zeros(max(self.m, 1))
        check(lib().pdhcg_get_scaling(self.handle, _dp(D), _dp(E)), "pdhcg_get_scaling")
        return D, E[: self.m]

    def phase_times(self):
        t = np.zeros(8)
        check(lib().pdhcg_get_phase_times(self.handle, _dp(t)), "pdhcg_get_phase_times")
        names = ["phase1", "inner_rows", "inner_elem", "phase2", "check", "barrier", "restart", "other"]
        return dict(zip(names, t.tolist()))

    def device(self):
        d = C.c_int32()
        check(lib().pdhcg_get_device(self.handle, C.byref(d)), "pdhcg_get_device")
        return int(d.value)

    def device_bytes(self):
        n, m, b = C.c_int32(), C.c_int32(), C.c_size_t()
        check(lib().pdhcg_get_info(self.handle, C.byref(n), C.byref(m), C.byref(b)), "pdhcg_get_info")
        return int(b.value)

    def close(self):
        if getattr(self, "handle", None):
            lib().pdhcg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _problem_table(qps):
    """The pdhcg_problem_data array of qps (with the buffers it points into)."""
    holds = [_qp_args(q) for q in qps]
    addr = np.array([(C.addressof(h["Q"].s) if "Q" in h else 0, C.addressof(h["A"].s), h["c"].ctypes.data,
                      h["lc"].ctypes.data if h["lc"].size else 0, h["uc"].ctypes.data if h["uc"].size else 0,
                      h["lv"].ctypes.data, h["uv"].ctypes.data) for h in holds],
                    dtype=np.uint64).reshape(len(qps), 7)
    assert C.sizeof(ProblemData) == 7 * 8
    return holds, addr


def autotune(qps, params: Params | None = None, stream=None):
    """pdhcg_autotune: time the row-layout and launch-shape candidates on qps
    (one problem: a single solve; several: a batched launch) and return
    (params with the chosen settings, report dict)."""
    p = Params()
    C.memmove(C.byref(p), C.byref(params if params is not None else default_params()), C.sizeof(Params))
    holds, addr = _problem_table(qps)
    t = Tuning()
    check(lib().pdhcg_autotune(len(qps), addr.ctypes.data_as(C.POINTER(ProblemData)), C.byref(p),
                               _P(stream) if stream else None, C.byref(t)), "pdhcg_autotune")
    return p, {k: getattr(t, k) for k, _ in t._fields_}


def create_batch(qps, params: Params | None = None, stream=None):
    """Create many Problems at once (pdhcg_create_batch: shared allocation, one setup launch)."""
    if any(getattr(q, "R", None) is not None for q in qps):
        raise ValueError("create_batch takes plain Q; create structured (Q + R^T R) problems one by one")
    params = params if params is not None else default_params()
    # the pdhcg_problem_data array: seven pointers per problem, filled as integers
    holds, addr = _problem_table(qps)
    data = addr.ctypes.data_as(C.POINTER(ProblemData))
    handles = (_P * len(qps))()
    check(lib().pdhcg_create_batch(len(qps), data, C.byref(params), _P(stream) if stream else None,
                                   handles), "pdhcg_create_batch")
    return [Problem(q, params, _handle=_P(handles[i])) for i, q in enumerate(qps)]


def solve_batch(problems, want_solutions=True):
    """Solve many Problems in one persistent launch (pdhcg_solve_batch)."""
    count = len(problems)
    handles = (_P * count)(*[p.handle for p in problems])
    res = (Result * count)()
    xs = [np.zeros(p.n) for p in problems] if want_solutions else None
    ys = [np.zeros(max(p.m, 1)) for p in problems] if want_solutions else None
    # the double* tables as integer address arrays (one cast each, not one per problem)
    xa = np.array([x.ctypes.data for x in xs], dtype=np.uint64) if want_solutions else None
    ya = np.array([y.ctypes.data for y in ys], dtype=np.uint64) if want_solutions else None
    xp = xa.ctypes.data_as(C.POINTER(_D)) if want_solutions else None
    yp = ya.ctypes.data_as(C.POINTER(_D)) if want_solutions else None
    check(lib().pdhcg_solve_batch(handles, count, res, xp, yp), "pdhcg_solve_batch")
    out = [r.as_dict() for r in res]
    if want_solutions:
        return [(xs[i], ys[i][: problems[i].m], out[i]) for i in range(count)]
    return out


NOALLOC_MAX_INSTANCES = 1024  # PDHCG_NOALLOC_MAX_INSTANCES


def check_noalloc_outputs(problems, x_out, y_out, device=None):
    """Validate the caller's output tensors before the kernel writes into them.

    Each list has one entry per problem; a non-None entry must be a contiguous
    float64 CUDA tensor on ``device`` (the handles' device, if given) with at
    least n_i (x) or m_i (y) elements.  Raises ValueError otherwise: the kernel
    writes through the raw pointers, so a short, strided, wrongly typed or
    foreign-device buffer would be an out-of-bounds device write."""
    count = len(problems)
    for name, outs, size in (("x_out", x_out, lambda p: p.n), ("y_out", y_out, lambda p: p.m)):
        if outs is None:
            continue
        if len(outs) != count:
            raise ValueError(f"{name}: {len(outs)} entries for {count} problems")
        for i, (p, t) in enumerate(zip(problems, outs)):
            if t is None:
                continue
            if getattr(t, "dtype", None) is None or str(t.dtype) != "torch.float64":
                raise ValueError(f"{name}[{i}]: dtype must be torch.float64, got {getattr(t, 'dtype', None)}")
            if not t.is_contiguous():
                raise ValueError(f"{name}[{i}]: must be contiguous")
            if t.numel() < size(p):
                raise ValueError(f"{name}[{i}]: {t.numel()} elements, needs {size(p)}")
            if not getattr(t, "is_cuda", False):
                raise ValueError(f"{name}[{i}]: must be a CUDA tensor")
            if device is not None and t.device.index != device:
                raise ValueError(f"{name}[{i}]: on cuda:{t.device.index}, the problems are on cuda:{device}")


def solve_batch_noalloc(problems, x_out=None, y_out=None):
    """pdhcg_solve_batch_noalloc: the batched solve with static device scratch.

    ``x_out`` / ``y_out``: lists of float64 CUDA tensors (n_i / m_i elements; an
    entry may be None), or None; checked by check_noalloc_outputs.  Returns the
    result dicts."""
    count = len(problems)
    if count and (x_out is not None or y_out is not None):
        check_noalloc_outputs(problems, x_out, y_out, problems[0].device())
    handles = (_P * max(count, 1))(*[p.handle for p in problems])
    res = (Result * max(count, 1))()
    ptr = (lambda t: _P(t.data_ptr()) if t is not None else None)
    xp = (_P * count)(*[ptr(t) for t in x_out]) if x_out is not None else None
    yp = (_P * count)(*[ptr(t) for t in y_out]) if y_out is not None else None
    check(lib().pdhcg_solve_batch_noalloc(handles, count, res, xp, yp), "pdhcg_solve_batch_noalloc")
    return [res[i].as_dict() for i in range(count)]


class Server:
    """Continuous-batching serving loop (pdhcg_server_*)."""

    def __init__(self, hbm_budget_bytes: int, max_slots: int, params: Params | None = None, stream=None):
        self.params = params if params is not None else default_params()
        h = _P()
        check(lib().pdhcg_server_create(C.c_size_t(hbm_budget_bytes), int(max_slots), C.byref(self.params),
                                        _P(stream) if stream else None, C.byref(h)), "pdhcg_server_create")
        self.handle = h
        self.sizes = {}

    def submit(self, qp):
        h = _qp_args(qp)
        t = C.c_uint64()
        check(lib().pdhcg_submit(self.handle, C.byref(h["Q"].s) if "Q" in h else None, C.byref(h["A"].s),
                                 _dp(h["c"]), _dp(h["lc"]), _dp(h["uc"]), _dp(h["lv"]), _dp(h["uv"]),
                                 C.byref(t)), "pdhcg_submit")
        self.sizes[t.value] = (int(qp.n), int(qp.m))
        return t.value

    def poll(self, ticket):
        """None while pending, else (x, y, result dict)."""
        n, m = self.sizes[ticket]
        x = np.zeros(n)
        y = np.zeros(max(m, 1))
        res = Result()
        rc = check(lib().pdhcg_poll(self.handle, C.c_uint64(ticket), C.byref(res), _dp(x), _dp(y)), "pdhcg_poll")
        if rc == PENDING:
            return None
        del self.sizes[ticket]
        return x, y[:m], res.as_dict()

    def stats(self):
        st = ServerStats()
        check(lib().pdhcg_server_get_stats(self.handle, C.byref(st)), "pdhcg_server_get_stats")
        return {k: getattr(st, k) for k, _ in st._fields_}

    def close(self):
        if getattr(self, "handle", None):
            lib().pdhcg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def strerror(code):
    return lib().pdhcg_strerror(code).decode()
