"""GPU: launch shapes away from the defaults, and the wall-clock limit.

* Strip widths: the two-pivot kernels at grid sizes whose last column strip
  is partial (and, at 2048^2 in the dual form, the 115 strips of 36 columns
  that once ran without end: the selection read the pivot rows' rhs entries
  from the tableau while the CTA owning the rhs column could still be
  writing them) give the oracle's pivots and bits.
* time_limit_s: past the limit the host raises the abort word, every pivot
  kernel stops within a pass, the solve ends in LP_TIMEOUT, the handle
  refuses to resume until the LP is loaded again, and the reloaded solve is
  the oracle's.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library
from test_gpu_parity import Run, _oracle, assert_same

pytestmark = pytest.mark.gpu

MAX_LE, MIN_GE = capi.LP_MAX_LE, capi.LP_MIN_GE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _strips(P, ctas, vw=2, sector=4, nu=768):
    """(CTAs launched, strip width, width of the last strip) for a requested
    grid, by the launch-shape rule of the pipelined kernels."""
    g = max(ctas, -(-P // (nu * vw)), 1)
    w = -(-P // g)
    w = -(-w // sector) * sector
    G = -(-P // w)
    return G, w, P - (G - 1) * w


@pytest.mark.parametrize("zero_skip", [0, 2])
@pytest.mark.parametrize("ctas", [5, 13, 29, 57, 100, 120, 150])
@pytest.mark.parametrize("sense,pipeline", [(MIN_GE, 4), (MIN_GE, 1), (MAX_LE, 4), (MAX_LE, 5)])
def test_two_pivot_kernels_at_partial_last_strips(ctas, sense, pipeline, zero_skip):
    """zero_skip=0: contiguous strips, the last one partial; zero_skip=2: two
    runs per CTA, uneven by up to a sector, vectors left in place."""
    A, b, c = lpgen.dense_lp(300, 500, seed=ctas)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    m, n = A.shape
    P = -(-(n + m + 1) // 32) * 32
    G, w, last = _strips(P, ctas)
    assert 0 < last <= w
    assert_same(Run(A, b, c, sense, ctas=ctas, pipeline=pipeline, zero_skip=zero_skip,
                    time_limit_s=60.0),
                _oracle(A, b, c, sense))


@pytest.mark.parametrize("ctas", [120, 94, 74])
def test_dual_2048_at_narrow_grids(ctas):
    """The 2048^2 dual form on 115 CTAs of 36-column strips (ctas=120) and on
    two other grids of the launch-shape sweep, under a wall-clock guard."""
    A, b, c = lpgen.dual_of(*lpgen.dense_lp(2048, 2048, seed=0))
    g = Run(A, b, c, MIN_GE, ctas=ctas, time_limit_s=120.0)
    assert g.status == capi.LP_OPTIMAL
    assert_same(g, _oracle(A, b, c, MIN_GE))


@pytest.mark.parametrize("precision,sense,pipeline", [
    (capi.LP_FP64, MAX_LE, 0), (capi.LP_FP64, MAX_LE, 2), (capi.LP_FP64, MAX_LE, 3),
    (capi.LP_FP64, MAX_LE, 4), (capi.LP_FP64, MAX_LE, 5), (capi.LP_FP64, MIN_GE, 1),
    (capi.LP_FP64, MIN_GE, 2), (capi.LP_FP32_REINV, MAX_LE, 1)])
def test_time_limit_ends_in_timeout_and_reload_solves(precision, sense, pipeline):
    # the paper's own random family at 1024^2, seed 1: 365 pivots, milliseconds
    A, b, c = lpgen.paper_lp(1024, 1024, seed=1)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    o = oracle.solve(A, b, c, sense=sense)
    h = capi.lp_create(capi.lp_options_default(precision=precision, pipeline=pipeline,
                                               time_limit_s=2e-4))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        _, st, it = capi.lp_result(h)
        assert st == capi.LP_TIMEOUT and it < o.iters
        with pytest.raises(capi.LpError) as e:
            capi.lp_solve(h)
        assert e.value.code == capi.LP_ERR_STATE
    finally:
        capi.lp_destroy(h)
    # a fresh load on a handle without a limit, in the same process
    h = capi.lp_create(capi.lp_options_default(precision=precision, pipeline=pipeline))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        obj, st, it = capi.lp_result(h)
        assert st == capi.LP_OPTIMAL
        if precision == capi.LP_FP64:
            assert it == o.iters and obj == o.obj
        else:
            assert abs(obj - o.obj) <= 1e-6 * abs(o.obj)
    finally:
        capi.lp_destroy(h)


def test_time_limit_same_handle_reload():
    # the paper's family at 2048^2, seed 1: 24734 pivots, about half a second
    A, b, c = lpgen.paper_lp(2048, 2048, seed=1)
    h = capi.lp_create(capi.lp_options_default(time_limit_s=2e-3))
    try:
        capi.lp_load(h, A, b, c)
        capi.lp_solve(h)
        assert capi.lp_result(h)[1] == capi.LP_TIMEOUT
        A2, b2, c2 = lpgen.dense_lp(5, 3, seed=3)  # a tiny LP finishes well inside the limit
        o2 = oracle.solve(A2, b2, c2)
        capi.lp_load(h, A2, b2, c2)
        capi.lp_solve(h)
        obj, st, it = capi.lp_result(h)
        assert st == capi.LP_OPTIMAL and it == o2.iters and obj == o2.obj
    finally:
        capi.lp_destroy(h)
