"""GPU: split runs and vectors left in place in the two-pivot primal kernel.

With lp_options.zero_skip (the default) every CTA of the FP64 two-pivot primal
kernel owns a run of the structural columns and a run of the slack and rhs
columns, and a pass leaves in place the column vectors whose entries in both
its pivot rows are zeros, their rows staying in whichever tableau buffer holds
them.  Sec. 2 Step 5 updates every entry with one fma per pivot; with a zero
multiplier that fma returns the entry itself unless the entry is -0, so the
kernel must leave every pivot and every bit of the tableau (signed zeros
included) as the oracle's: at grids whose runs are uneven, with -0 in the data
(where nothing may be left in place), with entries that round to -0 during the
solve, in both forms and with the option off.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library
from test_gpu_parity import Run, _bits, _oracle, assert_same

pytestmark = pytest.mark.gpu

MAX_LE, MIN_GE = capi.LP_MAX_LE, capi.LP_MIN_GE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


@pytest.mark.parametrize("zero_skip", [0, 2])
@pytest.mark.parametrize("sense,pipeline", [(MAX_LE, 4), (MAX_LE, 5), (MIN_GE, 4)])
@pytest.mark.parametrize("m,n,ctas", [(300, 500, 0), (500, 300, 0), (300, 500, 37),
                                      (257, 1000, 150), (1000, 257, 7), (64, 2048, 0),
                                      (2048, 64, 0)])
def test_split_strips_bitwise(m, n, ctas, sense, pipeline, zero_skip):
    A, b, c = lpgen.dense_lp(m, n, seed=m + 7 * n)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    assert_same(Run(A, b, c, sense, ctas=ctas, pipeline=pipeline, zero_skip=zero_skip,
                    time_limit_s=60.0),
                _oracle(A, b, c, sense))


def _sparse_signed(m, n, negzero, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(1, 100, size=(m, n)).astype(np.float64)
    A[rng.random((m, n)) < 0.5] = -0.0 if negzero else 0.0
    for j in range(n):
        if not np.any(A[:, j] > 0):
            A[rng.integers(0, m), j] = 1.0
    b = rng.integers(100, 10000, size=m).astype(np.float64)
    c = rng.integers(1, 50, size=n).astype(np.float64)
    return A, b, c


@pytest.mark.parametrize("negzero", [False, True])
@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
def test_signed_zeros_both_forms(negzero, sense):
    """Half of A zero, stored as +0 or as -0: long zero runs in the pivot rows
    of both forms; with -0 in the data nothing may be left in place (an fma
    with a zero multiplier turns some -0 entries into +0)."""
    A, b, c = _sparse_signed(600, 800, negzero, seed=5)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    o = _oracle(A, b, c, sense)
    assert o.status in (oracle.OPTIMAL, oracle.UNBOUNDED, oracle.INFEASIBLE)
    for pipeline in (1, 4):
        assert_same(Run(A, b, c, sense, pipeline=pipeline, zero_skip=2), o)


def _solve_counts(A, b, c, sense, **opts):
    h = capi.lp_create(capi.lp_options_default(**opts))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        obj, st, it = capi.lp_result(h)
        f, z = capi.lp_update_counts(h)
    finally:
        capi.lp_destroy(h)
    return obj, st, it, f, z


def test_update_counts_cover_the_tableau():
    """Every pivot either updates or leaves in place each vector of the m
    constraint rows over the whole row pitch; with the option off every one
    is updated.  A dense LP with few pivots relative to m keeps most slack
    columns at their unit vectors, so most of them stay in place."""
    sense = MAX_LE
    A, b, c = lpgen.dense_lp(1024, 1024, seed=3)
    m, n = A.shape
    P = (n + m + 1 + 31) // 32 * 32
    obj1, st1, it1, f1, z1 = _solve_counts(A, b, c, sense, pipeline=4, zero_skip=2)
    obj0, st0, it0, f0, z0 = _solve_counts(A, b, c, sense, pipeline=4, zero_skip=0)
    assert st1 == st0 == capi.LP_OPTIMAL
    assert it1 == it0 and obj1 == obj0
    assert f1 + z1 == it1 * P * m
    assert f0 == it0 * P * m and z0 == 0
    assert z1 > 0.3 * (f1 + z1), (f1, z1)


def test_fp32_same_bits_with_and_without():
    """FP32 mode (vectors left in place between its refreshes, each launch
    first finding the vectors that hold a -0) gives the same bits with the
    option forced on and off."""
    A, b, c = lpgen.dense_lp(1024, 1536, seed=11)
    out = []
    for zs in (2, 0):
        h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, zero_skip=zs))
        try:
            capi.lp_load(h, A, b, c)
            capi.lp_solve(h)
            x = np.empty(A.shape[1])
            y = np.empty(A.shape[0])
            obj, st, it = capi.lp_result(h, x, y)
        finally:
            capi.lp_destroy(h)
        out.append((obj, st, it, _bits(x), _bits(y)))
    (o1, s1, i1, x1, y1), (o0, s0, i0, x0, y0) = out
    assert s1 == s0 == capi.LP_OPTIMAL and i1 == i0
    assert _bits([o1])[0] == _bits([o0])[0]
    assert np.array_equal(x1, x0) and np.array_equal(y1, y0)


def test_entries_rounding_to_negative_zero():
    """Entries of -2^-1074 (the smallest subnormal, negated) in A: the first
    pivot row holds one, and dividing it by the pivot rounds it to -0 (the
    oracle's tableau after one pivot shows it), so from then on the kernel
    may not leave that vector in place.  Every bit as the oracle's after the
    first pivot and at the end."""
    A, b, c = lpgen.dense_lp(700, 900, seed=21)
    rng = np.random.default_rng(4)
    A[rng.integers(0, 700, 400), rng.integers(0, 900, 400)] = -5e-324
    o1 = _oracle(A, b, c, max_iters=1)
    assert (_bits(o1.T[:-1].ravel()) == 0x8000000000000000).any()
    assert_same(Run(A, b, c, pipeline=4, max_iters=1, zero_skip=2), o1)
    assert_same(Run(A, b, c, pipeline=4, zero_skip=2), _oracle(A, b, c))


def test_default_size_rule():
    """By default (zero_skip 1) vectors stay in place only on tableaus of at
    least 2^25 elements: 4096^2 (4097 x 8224) does, 1024^2 does not; every
    bit as the oracle's at 4096^2."""
    A, b, c = lpgen.dense_lp(4096, 4096, seed=7)
    o = _oracle(A, b, c)
    g = Run(A, b, c)
    assert_same(g, o)
    _, st, it, f, z = _solve_counts(A, b, c, MAX_LE)
    assert st == o.status and it == o.iters and z > 0.3 * (f + z)
    A, b, c = lpgen.dense_lp(1024, 1024, seed=3)
    assert _solve_counts(A, b, c, MAX_LE, pipeline=4)[4] == 0


def test_wide_lp_keeps_one_strip():
    """By default, below one slack column per four structural ones the runs
    are not split (few vectors would stay in place), even above the size
    threshold: 2048 x 16384 (2049 x 18464 elements); the oracle's bits."""
    A, b, c = lpgen.dense_lp(2048, 16384, seed=2)
    o = _oracle(A, b, c)
    _, st, it, f, z = _solve_counts(A, b, c, MAX_LE)
    assert st == o.status and it == o.iters and z == 0
    assert_same(Run(A, b, c), o)


def test_phase1_then_vectors_in_place():
    """Phase I (some b_i < 0): Phase 1 runs the dual rule (negative pivots
    write -0 entries), Phase 2 the primal kernel, which first finds the
    vectors holding a -0 and leaves only the others in place; the oracle's
    pivots and bits."""
    A, b, c = lpgen.dense_lp(300, 200, seed=1)
    A, b = lpgen.with_ge_rows(A, b, 0.1, seed=2)
    o = _oracle(A, b, c)
    assert o.status == oracle.OPTIMAL
    for pipeline in (1, 4, 5):
        assert_same(Run(A, b, c, pipeline=pipeline, zero_skip=2), o)


@pytest.mark.parametrize("e", [70, 130])
def test_scaled_lps_in_place(e):
    """Rows and columns scaled by 2^+-e (quotients outside the screening
    window, entries near the ends of the FP64 range): the oracle's bits."""
    from test_gpu_scaled import scaled_lp
    (A, b, c), eps, _ = scaled_lp(120, 150, e, seed=e)
    o = _oracle(A, b, c, **eps)
    assert o.status == oracle.OPTIMAL
    assert_same(Run(A, b, c, pipeline=4, zero_skip=2, **eps), o)


@pytest.mark.parametrize("chunk", [1, 7, 64])
def test_resumed_in_chunks(chunk):
    """Solves of a few pivots per call: each launch starts from one buffer,
    leaves vectors in the other and hands one buffer back; the oracle's
    pivots and bits after every call's worth, at the end."""
    A, b, c = lpgen.dense_lp(700, 900, seed=13)
    o = _oracle(A, b, c)
    m, n = A.shape
    h = capi.lp_create(capi.lp_options_default(pipeline=4, zero_skip=2, max_iters=chunk,
                                               trace_cap=4096))
    try:
        capi.lp_load(h, A, b, c)
        for _ in range(100000):
            capi.lp_solve(h)
            x, y = np.empty(n), np.empty(m)
            obj, st, it = capi.lp_result(h, x, y)
            if st != capi.LP_ITER_LIMIT:
                break
        assert st == o.status and it == o.iters
        assert _bits([obj])[0] == _bits([o.obj])[0]
        assert np.array_equal(_bits(x), _bits(o.x)) and np.array_equal(_bits(y), _bits(o.y))
        assert np.array_equal(_bits(capi.lp_get_tableau(h, m, n)), _bits(o.T))
    finally:
        capi.lp_destroy(h)


def test_fp32_nearly_dependent_same_bits():
    """The nearly-dependent-rows family in FP32 mode (body refreshes and
    dual-rule recovery between the primal launches): the same bits with
    vectors left in place as without."""
    A, b, c = lpgen.nearly_dependent_lp(600, 600, seed=3)
    out = []
    for zs in (2, 0):
        h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, zero_skip=zs,
                                                   reinv_k=7))
        try:
            capi.lp_load(h, A, b, c)
            capi.lp_solve(h)
            x = np.empty(A.shape[1])
            obj, st, it = capi.lp_result(h, x)
        finally:
            capi.lp_destroy(h)
        out.append((_bits([obj])[0], st, it, _bits(x)))
    assert out[0][:3] == out[1][:3] and np.array_equal(out[0][3], out[1][3])
