"""FP64 CPU oracle for the dense tableau simplex -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The product library never
imports it and shares no code with it.

Contents (each cites what it follows):

* :func:`solve` -- the tableau simplex of Sec. 2, Steps 1-5 (plain C in
  ``simplex_oracle.c``), primal form (max c'x, Ax <= b, x >= 0) and dual form
  (min c'x, Ax >= b, x >= 0, solved by the dual simplex).
* :class:`OracleTableau` -- the same, one call at a time (resumable runs,
  tableau snapshots) for pivot-by-pivot comparisons.
* :func:`brute_force` -- exact optimum of a tiny LP by vertex enumeration
  (the definition of the LP optimum of Eq. 1: the best basic feasible point).
* :func:`certificate` -- primal/dual feasibility, duality gap and
  complementary slackness residuals of a claimed optimum.
* :func:`reinvert` -- the tableau for a given basis, computed directly as
  B^-1 [A I b] with an LU solve (the plain definition of the tableau the
  pivots produce), used to pin the FP32 path's FP64 reinversion.

Default tolerances (the paper is silent; same formula in the library):
``eps_d = 1e-9*max(1, max|c|)``, ``eps_p = 1e-9*max(1, max|A|)``,
``eps_r = 1e-9*max(1, max|b|)``.
"""
import ctypes
import itertools
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

from .build import build_oracle

OPTIMAL, UNBOUNDED, ITER_LIMIT, INFEASIBLE = 0, 1, 2, 3
STATUS_NAMES = {OPTIMAL: "optimal", UNBOUNDED: "unbounded", ITER_LIMIT: "iter_limit",
                INFEASIBLE: "infeasible"}
MAX_LE, MIN_GE = 0, 1

_lib = None


def _bind(lib):
    """Declare the C signatures on a loaded oracle library."""
    dp = ctypes.POINTER(ctypes.c_double)
    ip = ctypes.POINTER(ctypes.c_int)
    llp = ctypes.POINTER(ctypes.c_longlong)
    lib.oracle_build.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, ctypes.c_int, dp, ip]
    lib.oracle_build.restype = None
    lib.oracle_build_phase1.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, dp, dp, ip]
    lib.oracle_build_phase1.restype = None
    lib.oracle_phase2_objective.argtypes = [ctypes.c_int, ctypes.c_int, dp, ip, dp]
    lib.oracle_phase2_objective.restype = None
    lib.oracle_run.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip,
                               ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                               ctypes.c_longlong, llp, ip, ip, ip, ctypes.c_longlong]
    lib.oracle_run.restype = ctypes.c_int
    lib.oracle_extract.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, ip, dp, dp, dp]
    lib.oracle_extract.restype = None
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_set_threads.restype = None
    lib.oracle_max_threads.argtypes = []
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    if _lib is None:
        _lib = _bind(ctypes.CDLL(build_oracle()))
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int))


def set_threads(t: int) -> None:
    """Number of OpenMP threads for the Step 5 row loop (results do not change)."""
    _load().oracle_set_threads(int(t))


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def default_eps(A, b, c):
    """(eps_d, eps_p, eps_r) from the documented formula."""
    A = np.asarray(A, dtype=np.float64)
    amax = float(np.max(np.abs(A))) if A.size else 0.0
    cmax = float(np.max(np.abs(c))) if len(c) else 0.0
    bmax = float(np.max(np.abs(b))) if len(b) else 0.0
    return 1e-9 * max(1.0, cmax), 1e-9 * max(1.0, amax), 1e-9 * max(1.0, bmax)


@dataclass
class OracleResult:
    status: int
    obj: float
    x: np.ndarray
    y: np.ndarray
    iters: int
    trace_p: np.ndarray
    trace_q: np.ndarray
    basis: np.ndarray
    T: Optional[np.ndarray] = field(default=None, repr=False)

    @property
    def status_name(self) -> str:
        return STATUS_NAMES[self.status]


class OracleTableau:
    """Step 1 (Sec. 2) once, then any number of resumable pivot runs.

    The primal form with some b_i < 0 (not covered by the paper's Sec. 2)
    goes through Phase I: Phase 1 prices with c' = min(c, 0), whose slack
    basis is dual feasible, and runs the dual simplex until every rhs is
    >= -eps_r (or the LP proves infeasible); Phase 2 rebuilds the objective
    row for c in that basis (oracle_phase2_objective), restarts the
    degenerate-pivot count and runs the primal simplex.  Pivots are counted
    and traced across both phases."""

    def __init__(self, A, b, c, sense=MAX_LE, eps_d=None, eps_p=None, eps_r=None,
                 bland_after=32, trace_cap=0):
        A = np.ascontiguousarray(A, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        c = np.ascontiguousarray(c, dtype=np.float64)
        m, n = A.shape
        assert b.shape == (m,) and c.shape == (n,)
        if sense == MIN_GE and np.any(c < 0):
            raise ValueError("dual form needs c >= 0 (slack basis dual feasible)")
        d, p, r = default_eps(A, b, c)
        self.eps_d = d if eps_d is None else float(eps_d)
        self.eps_p = p if eps_p is None else float(eps_p)
        self.eps_r = r if eps_r is None else float(eps_r)
        self.m, self.n, self.sense = m, n, sense
        self.bland_after = int(bland_after)
        self.T = np.empty((m + 1, n + m + 1), dtype=np.float64)
        self.basis = np.empty(m, dtype=np.int32)
        self.c = c
        # 0: no Phase I; 1: Phase 1 (dual simplex on c' = min(c, 0)); 2: Phase 2
        self.phase = 1 if sense == MAX_LE and np.any(b < 0) else 0
        if self.phase:
            _load().oracle_build_phase1(m, n, _dp(A), _dp(b), _dp(c), _dp(self.T), _ip(self.basis))
        else:
            _load().oracle_build(m, n, _dp(A), _dp(b), _dp(c), sense, _dp(self.T), _ip(self.basis))
        self.iters = ctypes.c_longlong(0)
        self.deg = ctypes.c_int(0)
        self.trace_cap = int(trace_cap)
        self.trace_p = np.full(max(self.trace_cap, 1), -1, dtype=np.int32)
        self.trace_q = np.full(max(self.trace_cap, 1), -1, dtype=np.int32)
        self.status = None

    def _run_rule(self, rule, max_iters):
        tp = _ip(self.trace_p) if self.trace_cap else None
        tq = _ip(self.trace_q) if self.trace_cap else None
        st = _load().oracle_run(self.m, self.n, rule, _dp(self.T), _ip(self.basis),
                                self.eps_d, self.eps_p, self.eps_r, self.bland_after,
                                int(max_iters), ctypes.byref(self.iters), ctypes.byref(self.deg),
                                tp, tq, self.trace_cap)
        if st < 0:
            raise MemoryError("oracle scratch allocation failed")
        return st

    def run(self, max_iters: int = 10 ** 12) -> int:
        """Pivot until a terminal status or until `max_iters` pivots in total."""
        if self.phase == 1:
            st = self._run_rule(MIN_GE, max_iters)  # the dual simplex rule
            if st != OPTIMAL:  # INFEASIBLE, or ITER_LIMIT (resumable in Phase 1)
                self.status = st
                return st
            _load().oracle_phase2_objective(self.m, self.n, _dp(self.T), _ip(self.basis),
                                            _dp(self.c))
            self.phase = 2
            self.deg.value = 0
        st = self._run_rule(MAX_LE if self.phase else self.sense, max_iters)
        self.status = st
        return st

    def extract(self):
        x = np.empty(self.n, dtype=np.float64)
        y = np.empty(self.m, dtype=np.float64)
        obj = ctypes.c_double(0.0)
        _load().oracle_extract(self.m, self.n, self.sense, _dp(self.T), _ip(self.basis),
                               _dp(x), _dp(y), ctypes.byref(obj))
        return x, y, obj.value

    def result(self, keep_tableau=False) -> OracleResult:
        x, y, obj = self.extract()
        k = min(self.iters.value, self.trace_cap)
        return OracleResult(self.status, obj, x, y, self.iters.value,
                            self.trace_p[:k].copy(), self.trace_q[:k].copy(), self.basis.copy(),
                            self.T.copy() if keep_tableau else None)


def solve(A, b, c, sense=MAX_LE, eps_d=None, eps_p=None, eps_r=None, bland_after=32,
          max_iters=10 ** 12, trace_cap=0, keep_tableau=False, threads=None) -> OracleResult:
    """Solve one LP with the tableau simplex (Sec. 2, Steps 1-5)."""
    if threads is not None:
        set_threads(threads)
    t = OracleTableau(A, b, c, sense, eps_d, eps_p, eps_r, bland_after, trace_cap)
    t.run(max_iters)
    return t.result(keep_tableau)


def brute_force(A, b, c, tol=1e-9):
    """Exact optimum of max c'x, Ax <= b, x >= 0 by enumerating every vertex.

    A vertex is a feasible point where n linearly independent constraints of
    the m + n (rows of A, and x_j >= 0) hold with equality; for a bounded
    feasible LP the optimum is attained at one (fundamental theorem of LP).
    Returns (z*, x*) or (None, None) when no vertex is feasible.  Only for
    tiny m, n: it solves C(m+n, n) linear systems.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    m, n = A.shape
    G = np.vstack([A, -np.eye(n)])
    h = np.concatenate([b, np.zeros(n)])
    best, bestx = None, None
    scale = max(1.0, float(np.max(np.abs(G))), float(np.max(np.abs(h))))
    for rows in itertools.combinations(range(m + n), n):
        Gs = G[list(rows)]
        if np.linalg.matrix_rank(Gs) < n:
            continue
        x = np.linalg.solve(Gs, h[list(rows)])
        if np.all(G @ x <= h + tol * scale * max(1.0, float(np.max(np.abs(x))))):
            z = float(c @ x)
            if best is None or z > best:
                best, bestx = z, x
    return best, bestx


def certificate(A, b, c, x, y, obj, sense=MAX_LE):
    """Residuals of the optimality certificate of (x, y).

    Primal form: Ax <= b, x >= 0, A'y >= c, y >= 0, c'x = b'y = obj.
    Dual form (min c'x, Ax >= b): Ax >= b, x >= 0, A'y <= c, y >= 0,
    c'x = b'y = obj.  Complementary slackness: y_i (b - Ax)_i = 0 and
    x_j (A'y - c)_j = 0.  Returned values are >= 0 violations (0 is exact).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    Ax = A @ x
    Aty = A.T @ y
    if sense == MAX_LE:
        primal = max(0.0, float(np.max(Ax - b)) if len(b) else 0.0)
        dual = max(0.0, float(np.max(c - Aty)) if len(c) else 0.0)
    else:
        primal = max(0.0, float(np.max(b - Ax)) if len(b) else 0.0)
        dual = max(0.0, float(np.max(Aty - c)) if len(c) else 0.0)
    return {
        "primal_infeas": primal,
        "x_neg": max(0.0, float(-np.min(x)) if len(x) else 0.0),
        "dual_infeas": dual,
        "y_neg": max(0.0, float(-np.min(y)) if len(y) else 0.0),
        "gap": abs(float(c @ x) - float(b @ y)),
        "obj_vs_cx": abs(float(c @ x) - obj),
        "compl_rows": float(np.max(np.abs(y * (b - Ax)))) if len(b) else 0.0,
        "compl_cols": float(np.max(np.abs(x * (Aty - c)))) if len(c) else 0.0,
    }


def reinvert(A, b, c, basis, sense=MAX_LE):
    """Tableau of basis `basis` (basic variable of each row) from the data.

    With D = [A I] (or [-A I] for the dual form), rhs = b (or -b) and
    objective coefficients chat = c (or -c) padded with zeros for slacks, the
    tableau the pivots reach is rows B^-1 [D | rhs] with B = D[:, basis], and
    objective row [-chat | 0] + chat_B' B^-1 [D | rhs].  Plain FP64 with a
    library LU solve.
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    c = np.asarray(c, dtype=np.float64)
    m, n = A.shape
    sgn = 1.0 if sense == MAX_LE else -1.0
    D = np.hstack([sgn * A, np.eye(m), (sgn * b)[:, None]])
    chat = np.concatenate([sgn * c, np.zeros(m)])
    basis = np.asarray(basis)
    B = D[:, basis]
    rows = np.linalg.solve(B, D)
    obj = np.concatenate([-chat, [0.0]]) + chat[basis] @ rows
    return np.vstack([rows, obj[None, :]])
