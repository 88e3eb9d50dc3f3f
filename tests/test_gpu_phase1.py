"""Phase I through the C ABI (the primal form with some b_i < 0; not in the
paper): Phase 1 runs the dual simplex rule on the objective row
max(-c, 0), Phase 2 rebuilds the objective row for c and runs the primal
rule.  Every pivot, the final tableau and the solution equal the oracle's
bit for bit, in every kernel mode and across resumed calls.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu

MAX_LE = capi.LP_MAX_LE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _gpu(A, b, c, cap=4096, chunk=None, **opts):
    m, n = A.shape
    if chunk:
        opts["max_iters"] = chunk
    h = capi.lp_create(capi.lp_options_default(trace_cap=cap, **opts))
    try:
        capi.lp_load(h, A, b, c, MAX_LE)
        calls = 0
        while True:
            capi.lp_solve(h)
            calls += 1
            x, y = np.empty(n), np.empty(m)
            obj, st, it = capi.lp_result(h, x, y)
            if st != capi.LP_ITER_LIMIT or not chunk or calls > 100000:
                break
        tp, tq = capi.lp_get_trace(h, cap)
        return dict(obj=obj, status=st, iters=it, x=x, y=y, tp=tp, tq=tq,
                    basis=capi.lp_get_basis(h, m), T=capi.lp_get_tableau(h, m, n), calls=calls)
    finally:
        capi.lp_destroy(h)


def _same(g, o):
    assert g["status"] == o.status, (g["status"], o.status)
    assert g["iters"] == o.iters, (g["iters"], o.iters)
    assert np.array_equal(g["tp"], o.trace_p) and np.array_equal(g["tq"], o.trace_q)
    assert _bits([g["obj"]])[0] == _bits([o.obj])[0], (g["obj"], o.obj)
    assert np.array_equal(_bits(g["x"]), _bits(o.x))
    assert np.array_equal(_bits(g["y"]), _bits(o.y))
    assert np.array_equal(g["basis"], o.basis)
    assert np.array_equal(_bits(g["T"]), _bits(o.T))


def _case(m, n, frac, seed=1):
    A, b, c = lpgen.dense_lp(m, n, seed)
    A, b = lpgen.with_ge_rows(A, b, frac, seed=seed + 1)
    return A, b, c


_ORACLE = {}


def _oracle(A, b, c, key):
    if key not in _ORACLE:
        _ORACLE[key] = oracle.solve(A, b, c, trace_cap=4096, keep_tableau=True)
    return _ORACLE[key]


@pytest.mark.parametrize("pipeline", [0, 1, 2, 4, 5])
@pytest.mark.parametrize("m,n,frac", [(5, 4, 0.4), (40, 61, 0.1), (100, 300, 0.2), (300, 200, 0.1)])
def test_phase1_bitwise(m, n, frac, pipeline):
    """Phase 1 on each dual-rule kernel (pipeline 0: selection then update;
    2: one pivot per pass; 1, 4, 5: two per pass), Phase 2 on the primal
    kernel of the mode: the oracle's pivots and bits."""
    A, b, c = _case(m, n, frac)
    o = _oracle(A, b, c, (m, n, frac))
    assert o.status == oracle.OPTIMAL
    _same(_gpu(A, b, c, pipeline=pipeline), o)


@pytest.mark.parametrize("chunk", [1, 7, 64])
def test_phase1_resume_in_chunks(chunk):
    """Calls of a few pivots each, stopping inside Phase 1, at the switch and
    inside Phase 2, end where one call ends."""
    A, b, c = _case(100, 300, 0.2)
    o = _oracle(A, b, c, (100, 300, 0.2))
    g = _gpu(A, b, c, chunk=chunk)
    assert g["calls"] > 1
    _same(g, o)


def test_phase1_textbook():
    """max 2x1 + 3x2 s.t. x1 + x2 <= 4, x1 + x2 >= 2, x1 <= 3: z = 12 at
    x = (0, 4)."""
    A = np.array([[1.0, 1.0], [-1.0, -1.0], [1.0, 0.0]])
    b = np.array([4.0, -2.0, 3.0])
    c = np.array([2.0, 3.0])
    g = _gpu(A, b, c)
    assert g["status"] == capi.LP_OPTIMAL and g["obj"] == 12.0
    assert np.array_equal(g["x"], [0.0, 4.0])
    _same(g, oracle.solve(A, b, c, trace_cap=4096, keep_tableau=True))


@pytest.mark.parametrize("pipeline", [0, 1, 2])
def test_phase1_infeasible(pipeline):
    """A >= row that no x within the <= rows meets: LP_INFEASIBLE, with the
    oracle's pivots up to that point."""
    A, b, c = _case(60, 80, 0.2)
    b[np.argmin(b)] = -1e12
    o = oracle.solve(A, b, c, trace_cap=4096, keep_tableau=True)
    assert o.status == oracle.INFEASIBLE
    g = _gpu(A, b, c, pipeline=pipeline)
    assert g["status"] == capi.LP_INFEASIBLE
    _same(g, o)
    A2 = np.array([[1.0, 1.0], [1.0, 0.0]])
    g2 = _gpu(A2, np.array([-1.0, 3.0]), np.array([1.0, 1.0]), pipeline=pipeline)
    assert g2["status"] == capi.LP_INFEASIBLE and g2["iters"] == 0


def test_phase1_needs_fp64():
    """The FP32 mode has no Phase I: b < 0 is refused at load."""
    A, b, c = _case(20, 30, 0.2)
    h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV))
    try:
        with pytest.raises(capi.LpError) as e:
            capi.lp_load(h, A, b, c, MAX_LE)
        assert e.value.code == capi.LP_ERR_INFEASIBLE_START
    finally:
        capi.lp_destroy(h)
