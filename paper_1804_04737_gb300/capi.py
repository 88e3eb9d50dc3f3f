"""ctypes binding of the C ABI in ``include/gbsimplex.h`` (argument marshalling only).

Every function keeps the C name.  Arrays may be numpy arrays (host memory) or
torch tensors (host or CUDA memory); they are passed as raw pointers, so they
must be C-contiguous float64 (int32 for index outputs).  Errors raise
:class:`LpError` carrying the C error code and the library's message.

The CUDA library must have been built (``paper_1804_04737_gb300.build``); a
missing library raises instead of falling back to anything else.
"""
import ctypes
import os
from dataclasses import dataclass
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libgbsimplex.so")

LP_OK, LP_ERR_INVALID_ARG, LP_ERR_OOM, LP_ERR_CUDA, LP_ERR_INFEASIBLE_START, LP_ERR_STATE, \
    LP_ERR_BUSY = range(7)
LP_OPTIMAL, LP_UNBOUNDED, LP_ITER_LIMIT, LP_INFEASIBLE, LP_NUMERICAL, LP_TIMEOUT, \
    LP_NOT_SOLVED = range(7)
STATUS_NAMES = ["optimal", "unbounded", "iter_limit", "infeasible", "numerical", "timeout",
                "not_solved"]
LP_MAX_LE, LP_MIN_GE = 0, 1
LP_FP64, LP_FP32_REINV = 0, 1

_c_double_p = ctypes.POINTER(ctypes.c_double)


class lp_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("reinv_k", ctypes.c_int),
        ("max_iters", ctypes.c_longlong),
        ("eps_d", ctypes.c_double),
        ("eps_p", ctypes.c_double),
        ("eps_r", ctypes.c_double),
        ("bland_after", ctypes.c_int),
        ("threads", ctypes.c_int),
        ("spin_timeout_cycles", ctypes.c_longlong),
        ("cuda_stream", ctypes.c_void_p),
        ("device", ctypes.c_int),
        ("ctas", ctypes.c_int),
        ("trace_cap", ctypes.c_longlong),
        ("group_elems", ctypes.c_longlong),
        ("pipeline", ctypes.c_int),
        ("solo_elems", ctypes.c_longlong),
        ("time_limit_s", ctypes.c_double),
        ("reinv_body", ctypes.c_int),
        ("zero_skip", ctypes.c_int),
        ("spill_pivots", ctypes.c_longlong),
        ("lanes", ctypes.c_int),
    ]


class LpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("gbsimplex error %d: %s" % (code, msg))
        self.code = code


_lib = None

# (name, restype, argtypes) of every entry point of include/gbsimplex.h
_SIGS = [
    ("lp_options_default", None, [ctypes.POINTER(lp_options)]),
    ("lp_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(lp_options)]),
    ("lp_load", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int]),
    ("lp_solve", ctypes.c_int, [ctypes.c_void_p]),
    ("lp_solve_async", ctypes.c_int, [ctypes.c_void_p]),
    ("lp_result", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                 _c_double_p, ctypes.POINTER(ctypes.c_int),
                                 ctypes.POINTER(ctypes.c_longlong)]),
    ("lp_get_trace", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_longlong, ctypes.POINTER(ctypes.c_longlong)]),
    ("lp_get_basis", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("lp_get_tableau", ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    ("lp_kernel_time", ctypes.c_int, [ctypes.c_void_p, _c_double_p,
                                      ctypes.POINTER(ctypes.c_int)]),
    ("lp_solve_noalloc", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                        ctypes.POINTER(lp_options), ctypes.c_void_p,
                                        ctypes.c_void_p, _c_double_p,
                                        ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_longlong)]),
    ("lp_solve_batch", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.POINTER(lp_options),
                                      ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    ("lp_batch_stats", ctypes.c_int, [_c_double_p, ctypes.POINTER(ctypes.c_longlong),
                                      ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_int)]),
    ("lp_batch_autotune", ctypes.c_int, [ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                         ctypes.c_void_p, ctypes.POINTER(lp_options),
                                         ctypes.c_char_p, ctypes.POINTER(lp_options)]),
    ("lp_server_create", ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p),
                                        ctypes.POINTER(lp_options), ctypes.c_size_t,
                                        ctypes.c_int]),
    ("lp_server_submit", ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)]),
    ("lp_server_poll", ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong,
                                      ctypes.POINTER(ctypes.c_int), ctypes.c_void_p,
                                      ctypes.c_void_p, _c_double_p, ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong), _c_double_p]),
    ("lp_server_wait", ctypes.c_int, [ctypes.c_void_p, ctypes.c_ulonglong, ctypes.c_double,
                                      ctypes.c_void_p, ctypes.c_void_p, _c_double_p,
                                      ctypes.POINTER(ctypes.c_int),
                                      ctypes.POINTER(ctypes.c_longlong), _c_double_p]),
    ("lp_server_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_longlong),
                                       ctypes.POINTER(ctypes.c_size_t),
                                       ctypes.POINTER(ctypes.c_int)]),
    ("lp_server_spill_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_longlong),
                                             ctypes.POINTER(ctypes.c_size_t)]),
    ("lp_server_destroy", None, [ctypes.c_void_p]),
    ("lp_fp32_stats", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), _c_double_p,
                                     _c_double_p]),
    ("lp_update_counts", ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_longlong)]),
    ("lp_dgemm_emulated", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_void_p, ctypes.c_longlong, ctypes.c_void_p,
                                         ctypes.c_longlong, ctypes.c_void_p, ctypes.c_longlong,
                                         ctypes.POINTER(lp_options)]),
    ("lp_dgemm_stats", ctypes.c_int, [ctypes.POINTER(ctypes.c_longlong)]),
    ("lp_destroy", None, [ctypes.c_void_p]),
    ("lp_last_error", ctypes.c_char_p, [ctypes.c_void_p]),
    ("lp_version", ctypes.c_char_p, []),
    ("lp_options_size", ctypes.c_size_t, []),
]


def load_library(path: str = LIB_PATH):
    """Load the CUDA library (once) and declare its signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("gbsimplex CUDA library not built (%s); run "
                           "paper_1804_04737_gb300.build.build_library()" % path)
    lib = ctypes.CDLL(path)
    for name, res, args in _SIGS:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.lp_options_size() != ctypes.sizeof(lp_options):
        raise RuntimeError("lp_options layout mismatch between binding and library")
    _lib = lib
    return lib


def _check(code, h=None):
    if code != LP_OK:
        msg = load_library().lp_last_error(h)
        raise LpError(code, msg.decode() if msg else "")


def _ptr(a, dtype=np.float64):
    """Raw pointer of a contiguous numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr") and hasattr(a, "is_contiguous"):  # torch.Tensor
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        if str(a.dtype) != {np.float64: "torch.float64", np.int32: "torch.int32"}[dtype]:
            raise ValueError("tensor dtype must be %s" % np.dtype(dtype).name)
        return ctypes.c_void_p(a.data_ptr())
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be a C-contiguous %s numpy array" % np.dtype(dtype).name)
    return ctypes.c_void_p(a.ctypes.data)


def lp_options_default(**overrides) -> lp_options:
    o = lp_options()
    load_library().lp_options_default(ctypes.byref(o))
    for k, v in overrides.items():
        if k == "cuda_stream" and v is not None and not isinstance(v, int):
            v = v.cuda_stream  # torch.cuda.Stream
        setattr(o, k, v)
    return o


def lp_create(opt: Optional[lp_options] = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(load_library().lp_create(ctypes.byref(h), ctypes.byref(opt) if opt else None))
    return h


def lp_load(h, A, b, c, sense=LP_MAX_LE) -> None:
    m, n = int(A.shape[0]), int(A.shape[1])
    if tuple(b.shape) != (m,) or tuple(c.shape) != (n,):
        raise ValueError("shapes: A %s, b %s, c %s" % (tuple(A.shape), tuple(b.shape),
                                                       tuple(c.shape)))
    _check(load_library().lp_load(h, m, n, _ptr(A), _ptr(b), _ptr(c), int(sense)), h)


def lp_solve(h) -> None:
    _check(load_library().lp_solve(h), h)


def lp_solve_async(h) -> None:
    _check(load_library().lp_solve_async(h), h)


def lp_result(h, x=None, y=None):
    """(obj, status, iters); fills x and y when given."""
    obj = ctypes.c_double()
    st = ctypes.c_int()
    it = ctypes.c_longlong()
    _check(load_library().lp_result(h, _ptr(x), _ptr(y), ctypes.byref(obj), ctypes.byref(st),
                                    ctypes.byref(it)), h)
    return obj.value, st.value, it.value


def lp_get_trace(h, cap: int):
    rows = np.full(max(cap, 1), -1, dtype=np.int32)
    cols = np.full(max(cap, 1), -1, dtype=np.int32)
    cnt = ctypes.c_longlong()
    _check(load_library().lp_get_trace(h, _ptr(rows, np.int32), _ptr(cols, np.int32), cap,
                                       ctypes.byref(cnt)), h)
    return rows[:cnt.value], cols[:cnt.value]


def lp_get_basis(h, m: int):
    basis = np.empty(m, dtype=np.int32)
    _check(load_library().lp_get_basis(h, _ptr(basis, np.int32)), h)
    return basis


def lp_get_tableau(h, m: int, n: int):
    T = np.empty((m + 1, n + m + 1), dtype=np.float64)
    _check(load_library().lp_get_tableau(h, _ptr(T)), h)
    return T


def lp_kernel_time(h):
    """(milliseconds, launches) of the pivot kernel of the last solve."""
    ms = ctypes.c_double()
    n = ctypes.c_int()
    _check(load_library().lp_kernel_time(h, ctypes.byref(ms), ctypes.byref(n)), h)
    return ms.value, n.value


def _check_shape(a, shape, name):
    if a is not None and tuple(a.shape) != shape:
        raise ValueError("%s has shape %s, expected %s" % (name, tuple(a.shape), shape))


def lp_solve_noalloc(A, b, c, sense=LP_MAX_LE, opt: Optional[lp_options] = None, x=None,
                     y=None):
    """Allocation-free solve; returns (obj, status, iters) and fills x, y."""
    if len(A.shape) != 2:
        raise ValueError("A must be a matrix, got shape %s" % (tuple(A.shape),))
    m, n = int(A.shape[0]), int(A.shape[1])
    for a, shape, name in ((b, (m,), "b"), (c, (n,), "c"), (x, (n,), "x"), (y, (m,), "y")):
        _check_shape(a, shape, name)
    obj = ctypes.c_double()
    st = ctypes.c_int()
    it = ctypes.c_longlong()
    _check(load_library().lp_solve_noalloc(m, n, _ptr(A), _ptr(b), _ptr(c), int(sense),
                                           ctypes.byref(opt) if opt else None, _ptr(x), _ptr(y),
                                           ctypes.byref(obj), ctypes.byref(st),
                                           ctypes.byref(it)))
    return obj.value, st.value, it.value


def lp_fp32_stats(h):
    """(reinversions, reinversion ms, body-refresh ms) of the last FP32 solve."""
    n = ctypes.c_int()
    ms = ctypes.c_double()
    body = ctypes.c_double()
    _check(load_library().lp_fp32_stats(h, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(body)),
           h)
    return n.value, ms.value, body.value


def lp_update_counts(h):
    """(updated, left in place): constraint-row entries the two-pivot primal
    kernel updated and left in place, summed over the pivots since lp_load."""
    f = ctypes.c_longlong()
    z = ctypes.c_longlong()
    _check(load_library().lp_update_counts(h, ctypes.byref(f), ctypes.byref(z)), h)
    return f.value, z.value


def lp_dgemm_emulated(A, B, C, opt: Optional[lp_options] = None) -> None:
    """C = A B (FP64 device tensors, row-major) by emulated-FP64 tensor-core
    products; C must be an M x N float64 tensor on the device."""
    if len(A.shape) != 2 or len(B.shape) != 2 or len(C.shape) != 2:
        raise ValueError("A, B and C must be matrices")
    M, K = int(A.shape[0]), int(A.shape[1])
    if int(B.shape[0]) != K or tuple(C.shape) != (M, int(B.shape[1])):
        raise ValueError("shapes: A %s, B %s, C %s" % (tuple(A.shape), tuple(B.shape),
                                                       tuple(C.shape)))
    N = int(B.shape[1])
    for t in (A, B, C):
        if not hasattr(t, "is_cuda") or not t.is_cuda:
            raise ValueError("A, B and C must be device tensors")
    _check(load_library().lp_dgemm_emulated(M, N, K, _ptr(A), K, _ptr(B), N, _ptr(C), N,
                                            ctypes.byref(opt) if opt else None))


def lp_solve_batch(lps, opt: Optional[lp_options] = None, want_xy=False):
    """Solve a list of (A, b, c, sense) in one batched launch.

    A, b, c may be numpy arrays or (all) CUDA tensors.  Returns (obj, status,
    iters) arrays and, with want_xy, lists of x and y arrays."""
    k = len(lps)
    m = np.array([int(L[0].shape[0]) for L in lps], dtype=np.int32)
    n = np.array([int(L[0].shape[1]) for L in lps], dtype=np.int32)
    ptrs = [(_ptr(L[0]), _ptr(L[1]), _ptr(L[2])) for L in lps]
    Ap = (ctypes.c_void_p * k)(*[p[0].value for p in ptrs])
    bp = (ctypes.c_void_p * k)(*[p[1].value for p in ptrs])
    cp = (ctypes.c_void_p * k)(*[p[2].value for p in ptrs])
    sense = np.array([int(L[3]) if len(L) > 3 else LP_MAX_LE for L in lps], dtype=np.int32)
    obj = np.empty(k)
    st = np.empty(k, dtype=np.int32)
    it = np.empty(k, dtype=np.int64)
    xs = ys = None
    xp = yp = None
    if want_xy:
        xs = [np.empty(int(v)) for v in n]
        ys = [np.empty(int(v)) for v in m]
        xp = (ctypes.c_void_p * k)(*[a.ctypes.data for a in xs])
        yp = (ctypes.c_void_p * k)(*[a.ctypes.data for a in ys])
    _check(load_library().lp_solve_batch(k, m.ctypes.data, n.ctypes.data, Ap, bp, cp,
                                         sense.ctypes.data, ctypes.byref(opt) if opt else None,
                                         obj.ctypes.data, st.ctypes.data, it.ctypes.data, xp, yp))
    return (obj, st, it, xs, ys) if want_xy else (obj, st, it)


def lp_batch_autotune(lps, opt: Optional[lp_options] = None, cache_path=None) -> lp_options:
    """Fastest batched launch shape for this batch (see the C declaration)."""
    k = len(lps)
    m = np.array([int(L[0].shape[0]) for L in lps], dtype=np.int32)
    n = np.array([int(L[0].shape[1]) for L in lps], dtype=np.int32)
    ptrs = [(_ptr(L[0]), _ptr(L[1]), _ptr(L[2])) for L in lps]
    Ap = (ctypes.c_void_p * k)(*[p[0].value for p in ptrs])
    bp = (ctypes.c_void_p * k)(*[p[1].value for p in ptrs])
    cp = (ctypes.c_void_p * k)(*[p[2].value for p in ptrs])
    sense = np.array([int(L[3]) if len(L) > 3 else LP_MAX_LE for L in lps], dtype=np.int32)
    best = lp_options()
    _check(load_library().lp_batch_autotune(k, m.ctypes.data, n.ctypes.data, Ap, bp, cp,
                                            sense.ctypes.data,
                                            ctypes.byref(opt) if opt else None,
                                            cache_path.encode() if cache_path else None,
                                            ctypes.byref(best)))
    return best


def lp_batch_stats():
    """(kernel_ms, pivots, ctas, threads, max_group) of the last batched solve."""
    ms = ctypes.c_double()
    pv = ctypes.c_longlong()
    ct, th, mg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().lp_batch_stats(ctypes.byref(ms), ctypes.byref(pv), ctypes.byref(ct),
                                         ctypes.byref(th), ctypes.byref(mg)))
    return ms.value, pv.value, ct.value, th.value, mg.value


def lp_server_create(opt: Optional[lp_options] = None, hbm_budget_bytes=60 << 30,
                     max_slots=256):
    srv = ctypes.c_void_p()
    _check(load_library().lp_server_create(ctypes.byref(srv), ctypes.byref(opt) if opt else None,
                                           int(hbm_budget_bytes), int(max_slots)))
    return srv


def lp_server_submit(srv, A, b, c, sense=LP_MAX_LE) -> int:
    """Queue one LP (host arrays); returns its ticket."""
    t = ctypes.c_ulonglong()
    _check(load_library().lp_server_submit(srv, int(A.shape[0]), int(A.shape[1]), _ptr(A),
                                           _ptr(b), _ptr(c), int(sense), ctypes.byref(t)))
    return t.value


def _server_out(m, n):
    return (np.empty(n), np.empty(m), ctypes.c_double(), ctypes.c_int(), ctypes.c_longlong(),
            ctypes.c_double())


def lp_server_wait(srv, ticket, m, n, timeout_s=60.0):
    """(obj, status, iters, x, y, latency_ms) of a ticket, waiting for it."""
    x, y, obj, st, it, lat = _server_out(m, n)
    _check(load_library().lp_server_wait(srv, ticket, float(timeout_s), _ptr(x), _ptr(y),
                                         ctypes.byref(obj), ctypes.byref(st), ctypes.byref(it),
                                         ctypes.byref(lat)))
    return obj.value, st.value, it.value, x, y, lat.value


def lp_server_poll(srv, ticket, m, n):
    """None while pending, else (obj, status, iters, x, y, latency_ms)."""
    x, y, obj, st, it, lat = _server_out(m, n)
    done = ctypes.c_int()
    _check(load_library().lp_server_poll(srv, ticket, ctypes.byref(done), _ptr(x), _ptr(y),
                                         ctypes.byref(obj), ctypes.byref(st), ctypes.byref(it),
                                         ctypes.byref(lat)))
    return (obj.value, st.value, it.value, x, y, lat.value) if done.value else None


def lp_server_stats(srv):
    """(completed, kernel launches, HBM bytes in use, requests queued)."""
    c, l, q = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_int()
    u = ctypes.c_size_t()
    _check(load_library().lp_server_stats(srv, ctypes.byref(c), ctypes.byref(l), ctypes.byref(u),
                                          ctypes.byref(q)))
    return c.value, l.value, u.value, q.value


def lp_server_spill_stats(srv):
    """(LPs spilled to host memory, LPs readmitted, pinned host bytes held)."""
    sp, rs, hb = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t()
    _check(load_library().lp_server_spill_stats(srv, ctypes.byref(sp), ctypes.byref(rs),
                                                ctypes.byref(hb)))
    return sp.value, rs.value, hb.value


def lp_server_destroy(srv) -> None:
    if srv is not None:
        load_library().lp_server_destroy(srv)


def lp_destroy(h) -> None:
    if h is not None:
        load_library().lp_destroy(h)


def lp_last_error(h=None) -> str:
    msg = load_library().lp_last_error(h)
    return msg.decode() if msg else ""


def lp_version() -> str:
    return load_library().lp_version().decode()


@dataclass
class Result:
    status: int
    obj: float
    x: np.ndarray
    y: np.ndarray
    iters: int
    trace_p: Optional[np.ndarray] = None
    trace_q: Optional[np.ndarray] = None

    @property
    def status_name(self) -> str:
        return STATUS_NAMES[self.status]


def solve(A, b, c, sense=LP_MAX_LE, trace_cap=0, **opts) -> Result:
    """lp_create + lp_load + lp_solve + lp_result (+ lp_get_trace) + lp_destroy."""
    o = lp_options_default(trace_cap=trace_cap, **opts)
    h = lp_create(o)
    try:
        lp_load(h, A, b, c, sense)
        lp_solve(h)
        m, n = int(A.shape[0]), int(A.shape[1])
        x = np.empty(n, dtype=np.float64)
        y = np.empty(m, dtype=np.float64)
        obj, st, it = lp_result(h, x, y)
        tp = tq = None
        if trace_cap:
            tp, tq = lp_get_trace(h, trace_cap)
        return Result(st, obj, x, y, it, tp, tq)
    finally:
        lp_destroy(h)


def lp_dgemm_stats():
    """Tensor-core MMA instructions (128 x 64 x 16 bf16) the last
    lp_dgemm_emulated issued."""
    n = ctypes.c_longlong()
    _check(load_library().lp_dgemm_stats(ctypes.byref(n)))
    return n.value
