"""FP32 tableau with FP64 reinversion, through the C ABI.

The pivot sequence of FP32 pivoting is not required to match the FP64 oracle;
the bar is the objective within 1e-6 relative error of the FP64 oracle after
the final reinversion, and an FP64 optimality certificate.  The reinversion
itself (x_B = B^-1 b, duals, objective row, objective, for a given basis) is
pinned to the oracle's direct definition B^-1 [A I b] at intermediate bases.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu

MAX_LE, MIN_GE = capi.LP_MAX_LE, capi.LP_MIN_GE
OBJ_TOL = 1e-6


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _fp32(A, b, c, sense=MAX_LE, **opts):
    m, n = A.shape
    h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, **opts))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        x, y = np.empty(n), np.empty(m)
        obj, st, it = capi.lp_result(h, x, y)
        basis = capi.lp_get_basis(h, m)
        return obj, st, it, x, y, basis
    finally:
        capi.lp_destroy(h)


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


@pytest.mark.parametrize("m,n,sense", [(64, 64, MAX_LE), (300, 200, MAX_LE), (200, 300, MIN_GE),
                                       (2048, 2048, MAX_LE), (2048, 2048, MIN_GE),
                                       (512, 4096, MAX_LE), (4096, 512, MAX_LE)])
def test_fp32_objective_vs_fp64_oracle(m, n, sense):
    A, b, c = lpgen.dense_lp(m, n, seed=0)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    o = oracle.solve(A, b, c, sense=sense)
    obj, st, it, x, y, _ = _fp32(A, b, c, sense)
    assert st == capi.LP_OPTIMAL
    assert _rel(obj, o.obj) <= OBJ_TOL, (obj, o.obj)
    cert = oracle.certificate(A, b, c, x, y, obj, sense=sense)
    scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
    assert max(cert.values()) <= 1e-9 * scale * 1e3, cert


@pytest.mark.parametrize("k", [1, 7, 50, 200])
@pytest.mark.parametrize("pipeline", [0, 2, 3, 4, 5])
def test_fp32_reinversion_period(k, pipeline):
    A, b, c = lpgen.dense_lp(400, 500, seed=3)
    o = oracle.solve(A, b, c)
    obj, st, it, x, y, _ = _fp32(A, b, c, reinv_k=k, pipeline=pipeline)
    assert st == capi.LP_OPTIMAL and _rel(obj, o.obj) <= OBJ_TOL


@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
def test_reinversion_matches_definition_at_intermediate_bases(sense):
    """Stopped after k pivots, the reported FP64 x, y and objective are those
    of B^-1 [A I b] for the basis reached (oracle.reinvert)."""
    A, b, c = lpgen.dense_lp(120, 150, seed=4)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    m, n = A.shape
    total = oracle.solve(A, b, c, sense=sense).iters
    assert total >= 4
    for k in sorted({1, total // 2, total - 1}):
        obj, st, it, x, y, basis = _fp32(A, b, c, sense, max_iters=k, reinv_k=1000)
        assert st == capi.LP_ITER_LIMIT and it == k
        R = oracle.reinvert(A, b, c, basis, sense=sense)
        z = R[m, -1]
        assert _rel(obj, z if sense == MAX_LE else -z) <= 1e-9
        xr = np.zeros(n)
        for i, v in enumerate(basis):
            if v < n:
                xr[v] = R[i, -1]
        np.testing.assert_allclose(x, xr, rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(y, R[m, n:n + m], rtol=1e-9, atol=1e-9)


def test_fp32_small_klee_minty_and_textbook():
    for n in (2, 3, 4):
        A = np.zeros((n, n))
        bb = np.zeros(n)
        cc = np.zeros(n)
        for i in range(n):
            for j in range(i):
                A[i, j] = 2.0 * 10.0 ** (i - j)
            A[i, i] = 1.0
            bb[i] = 100.0 ** i
            cc[i] = 10.0 ** (n - 1 - i)
        obj, st, *_ = _fp32(A, bb, cc)
        assert st == capi.LP_OPTIMAL and _rel(obj, 100.0 ** (n - 1)) <= 1e-12
    obj, st, it, x, y, _ = _fp32(np.array([[1.0, 0], [0, 2], [3, 2]]), np.array([4.0, 12, 18]),
                                 np.array([3.0, 5]))
    assert st == capi.LP_OPTIMAL and obj == 36.0
    np.testing.assert_allclose(x, [2, 6], atol=1e-12)


def test_fp32_unbounded():
    obj, st, *_ = _fp32(np.array([[1.0, -1.0], [2.0, 0.0]]), np.array([4.0, 6.0]),
                        np.array([1.0, 3.0]))
    assert st == capi.LP_UNBOUNDED


@pytest.mark.parametrize("m,n,sense", [(512, 512, MAX_LE), (1024, 1024, MAX_LE), (1024, 1024, MIN_GE)])
def test_fp32_paper_family_objective(m, n, sense):
    """The paper's random family (real-valued data, which FP32 rounds; about
    1400 pivots at 1024^2): FP32 pivoting with FP64 reinversion still ends at
    the FP64 optimum within the tolerance, with an FP64 certificate."""
    A, b, c = lpgen.paper_lp(m, n, seed=2)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    o = oracle.solve(A, b, c, sense=sense)
    obj, st, it, x, y, _ = _fp32(A, b, c, sense)
    assert st == capi.LP_OPTIMAL
    assert _rel(obj, o.obj) <= OBJ_TOL, (obj, o.obj)
    cert = oracle.certificate(A, b, c, x, y, obj, sense=sense)
    scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
    assert max(cert.values()) <= 1e-9 * scale * 1e3, cert


@pytest.mark.parametrize("k", [50, 200])
def test_fp32_8192_objective_vs_oracle(k):
    """The 8192^2 dense LP of the bench: FP32 tableau with FP64 reinversion
    every k pivots, objective within 1e-6 of the FP64 oracle's, with an FP64
    certificate of the reported x and y."""
    A, b, c = lpgen.dense_lp(8192, 8192, seed=0)
    o = _oracle_8192()
    obj, st, it, x, y, _ = _fp32(A, b, c, reinv_k=k)
    assert st == capi.LP_OPTIMAL
    assert _rel(obj, o.obj) <= OBJ_TOL, (obj, o.obj)
    cert = oracle.certificate(A, b, c, x, y, obj)
    scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
    assert max(cert.values()) <= 1e-9 * scale * 1e3, cert


_O8192 = []


def _oracle_8192():
    if not _O8192:
        A, b, c = lpgen.dense_lp(8192, 8192, seed=0)
        _O8192.append(oracle.solve(A, b, c))
    return _O8192[0]
