"""GPU parity: the CUDA library against the FP64 oracle, through the C ABI.

FP64 mode follows the same arithmetic contract as the oracle, so the bar is
bit-for-bit equality of the pivot sequence, the final tableau, the objective,
x and y (stricter than the 1e-9 relative objective error the method needs).
"""
import os

import numpy as np
import pytest

import oracle
from golden_io import read_lp, read_table
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu

MAX_LE, MIN_GE = capi.LP_MAX_LE, capi.LP_MIN_GE


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


class Run:
    """One GPU solve with everything the parity checks look at."""

    def __init__(self, A, b, c, sense=MAX_LE, cap=4096, **opts):
        m, n = A.shape
        h = capi.lp_create(capi.lp_options_default(trace_cap=cap, **opts))
        try:
            capi.lp_load(h, A, b, c, sense)
            capi.lp_solve(h)
            self.x = np.empty(n)
            self.y = np.empty(m)
            self.obj, self.status, self.iters = capi.lp_result(h, self.x, self.y)
            self.tp, self.tq = capi.lp_get_trace(h, cap)
            self.basis = capi.lp_get_basis(h, m)
            self.T = capi.lp_get_tableau(h, m, n)
        finally:
            capi.lp_destroy(h)


def _oracle(A, b, c, sense=MAX_LE, cap=4096, **kw):
    return oracle.solve(A, b, c, sense=sense, trace_cap=cap, keep_tableau=True, **kw)


def assert_same(g, o, tableau=True):
    assert g.status == o.status, (g.status, o.status)
    assert g.iters == o.iters, (g.iters, o.iters)
    assert np.array_equal(g.tp, o.trace_p) and np.array_equal(g.tq, o.trace_q)
    assert _bits([g.obj])[0] == _bits([o.obj])[0], (g.obj, o.obj)
    assert np.array_equal(_bits(g.x), _bits(o.x))
    assert np.array_equal(_bits(g.y), _bits(o.y))
    assert np.array_equal(g.basis, o.basis)
    if tableau:
        assert np.array_equal(_bits(g.T), _bits(o.T))


SHAPES = [(64, 64), (1, 1), (1, 9), (9, 1), (5, 3), (33, 17), (100, 257), (257, 100),
          (300, 1000), (1000, 300)]


@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
@pytest.mark.parametrize("m,n", SHAPES)
def test_dense_bitwise(m, n, sense):
    A, b, c = lpgen.dense_lp(m, n, seed=m * 1000 + n)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    assert_same(Run(A, b, c, sense), _oracle(A, b, c, sense))


@pytest.mark.parametrize("ctas,threads", [(1, 64), (1, 1024), (2, 256), (3, 128), (7, 512),
                                          (40, 64), (0, 0)])
def test_launch_shapes_bitwise(ctas, threads):
    """The decomposition does not change a bit of the result."""
    A, b, c = lpgen.dense_lp(200, 311, seed=9)
    o = _oracle(A, b, c)
    assert_same(Run(A, b, c, ctas=ctas, threads=threads), o)
    Ad, bd, cd = lpgen.dual_of(A, b, c)
    od = _oracle(Ad, bd, cd, MIN_GE)
    assert_same(Run(Ad, bd, cd, MIN_GE, ctas=ctas, threads=threads), od)


@pytest.mark.parametrize("pipeline", [0, 2, 3, 4, 5])
@pytest.mark.parametrize("m,n,ctas,threads", [(1, 1, 0, 0), (9, 1, 0, 0), (33, 17, 2, 128),
                                              (257, 100, 0, 0), (300, 1000, 5, 256),
                                              (1000, 300, 0, 1024), (200, 311, 40, 64)])
def test_primal_kernels_bitwise(m, n, ctas, threads, pipeline):
    """Every primal kernel gives the oracle's pivots and bits: selection then
    update (0), pipelined in place (2), pipelined double-buffered (3), two
    pivots per pass (4), two pivots per pass with the ratio test distributed
    over the CTAs (5)."""
    A, b, c = lpgen.dense_lp(m, n, seed=7 * m + n)
    assert_same(Run(A, b, c, ctas=ctas, threads=threads, pipeline=pipeline), _oracle(A, b, c))


@pytest.mark.parametrize("pipeline", [0, 2, 3, 4, 5])
@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
def test_pivot_by_pivot_tableau(sense, pipeline):
    """One pivot per call: the tableau equals the oracle's after every pivot."""
    A, b, c = lpgen.dense_lp(40, 61, seed=12)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    m, n = A.shape
    t = oracle.OracleTableau(A, b, c, sense=sense)
    h = capi.lp_create(capi.lp_options_default(max_iters=1, ctas=4, threads=128,
                                               pipeline=pipeline))
    try:
        capi.lp_load(h, A, b, c, sense)
        for k in range(1, 500):
            capi.lp_solve(h)
            _, st, it = capi.lp_result(h)
            ost = t.run(max_iters=k)
            assert it == t.iters.value
            assert np.array_equal(_bits(capi.lp_get_tableau(h, m, n)), _bits(t.T)), k
            if st != capi.LP_ITER_LIMIT:
                assert st == ost == capi.LP_OPTIMAL
                break
            assert ost == oracle.ITER_LIMIT
        else:
            pytest.fail("did not finish")
    finally:
        capi.lp_destroy(h)


@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
@pytest.mark.parametrize("chunk,pipeline", [(7, 1), (1, 4), (2, 4), (3, 4), (7, 4), (5, 3), (1, 5), (3, 5)])
def test_resume_in_chunks(chunk, pipeline, sense):
    """Pivot limits that end a launch inside a two-pivot pass or between passes."""
    A, b, c = lpgen.dense_lp(150, 180, seed=13)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    o = _oracle(A, b, c, sense)
    h = capi.lp_create(capi.lp_options_default(max_iters=chunk, trace_cap=4096,
                                               pipeline=pipeline))
    try:
        capi.lp_load(h, A, b, c, sense)
        calls = 0
        while True:
            capi.lp_solve(h)
            calls += 1
            obj, st, it = capi.lp_result(h)
            if st != capi.LP_ITER_LIMIT:
                break
            assert it == chunk * calls
        tp, tq = capi.lp_get_trace(h, 4096)
        assert st == capi.LP_OPTIMAL and it == o.iters and obj == o.obj
        assert np.array_equal(tp, o.trace_p) and np.array_equal(tq, o.trace_q)
    finally:
        capi.lp_destroy(h)


def test_klee_minty_on_gpu():
    for n, pivots, z in read_table("klee_minty.txt"):
        n = int(n)
        A = np.zeros((n, n))
        b = np.zeros(n)
        c = np.zeros(n)
        for i in range(n):
            for j in range(i):
                A[i, j] = 2.0 * 10.0 ** (i - j)
            A[i, i] = 1.0
            b[i] = 100.0 ** i
            c[i] = 10.0 ** (n - 1 - i)
        g = Run(A, b, c)
        assert g.status == capi.LP_OPTIMAL and g.iters == int(pivots) and g.obj == z
        assert_same(g, _oracle(A, b, c))


@pytest.mark.parametrize("pipeline", [1, 4, 5])
@pytest.mark.parametrize("name", ["chvatal_cycling.txt", "beale_cycling.txt"])
def test_cycling_examples_on_gpu(name, pipeline):
    g0 = read_lp(name)
    A, b, c = g0["A"], g0["b"], g0["c"]
    g = Run(A, b, c, bland_after=10 ** 9, max_iters=60, cap=60, pipeline=pipeline)
    assert g.status == capi.LP_ITER_LIMIT and g.iters == 60
    assert_same(g, _oracle(A, b, c, bland_after=10 ** 9, max_iters=60, cap=60))
    for ba in (0, 1, 32):
        g = Run(A, b, c, bland_after=ba, pipeline=pipeline)
        assert g.status == capi.LP_OPTIMAL and abs(g.obj - g0["z"]) <= 1e-12
        assert_same(g, _oracle(A, b, c, bland_after=ba))


def test_bland_tie_trace_on_gpu():
    g0 = read_lp("bland_tie.txt")
    for ba, key in ((0, "bland"), (10 ** 9, "dantzig")):
        g = Run(g0["A"], g0["b"], g0["c"], bland_after=ba, cap=10)
        got = np.stack([g.tp, g.tq], axis=1).ravel()[:len(g0[key])]
        assert got.tolist() == g0[key].astype(int).tolist()
        assert g.obj == g0["z"]


def test_textbook_unbounded_infeasible_on_gpu():
    g0 = read_lp("wyndor.txt")
    g = Run(g0["A"], g0["b"], g0["c"])
    assert g.status == capi.LP_OPTIMAL and g.obj == g0["z"]
    assert np.array_equal(g.x, g0["x"]) and np.array_equal(g.y, g0["y"])
    g = Run(np.array([[1.0, -1.0], [2.0, 0.0]]), np.array([4.0, 6.0]), np.array([1.0, 3.0]))
    assert g.status == capi.LP_UNBOUNDED and g.iters == 0
    g = Run(np.array([[1.0, -1.0]]), np.array([2.0]), np.array([2.0, 1.0]))
    assert g.status == capi.LP_UNBOUNDED and g.iters == 1
    g = Run(np.array([[-1.0, -2.0]]), np.array([1.0]), np.array([1.0, 1.0]), MIN_GE)
    assert g.status == capi.LP_INFEASIBLE


@pytest.mark.parametrize("pipeline", [1, 4, 5])
def test_degenerate_integer_instances(pipeline):
    """Integer data with zeros in b: ties and degenerate pivots."""
    for seed in range(40):
        rng = np.random.default_rng(seed)
        m, n = (int(v) for v in rng.integers(2, 40, size=2))
        A = rng.integers(0, 4, size=(m, n)).astype(float)
        for j in range(n):
            if not np.any(A[:, j] > 0):
                A[rng.integers(0, m), j] = 1.0
        b = rng.integers(0, 3, size=m).astype(float)
        c = rng.integers(-1, 4, size=n).astype(float)
        for ba in (0, 3, 32):
            assert_same(Run(A, b, c, bland_after=ba, ctas=3, threads=64, pipeline=pipeline),
                        _oracle(A, b, c, bland_after=ba))


@pytest.mark.parametrize("m,n,sense", [(2048, 2048, MAX_LE), (2048, 2048, MIN_GE),
                                       (512, 4096, MAX_LE), (4096, 512, MAX_LE)])
def test_full_size_bitwise(m, n, sense):
    """The bench workload's LPs at full size, default launch shape."""
    A, b, c = lpgen.dense_lp(m, n, seed=0)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    g = Run(A, b, c, sense)
    o = _oracle(A, b, c, sense)
    assert g.status == capi.LP_OPTIMAL
    assert_same(g, o)


@pytest.mark.parametrize("m,n,pipeline", [(2048, 2048, 4), (4096, 512, 4), (512, 4096, 5)])
def test_full_size_two_pivot_passes(m, n, pipeline):
    """Two pivots per pass at full size; 4 takes the distributed ratio test
    for 2048 and 4096 rows and the per-CTA one for 512, 5 forces it."""
    A, b, c = lpgen.dense_lp(m, n, seed=0)
    assert_same(Run(A, b, c, pipeline=pipeline), _oracle(A, b, c))


@pytest.mark.parametrize("pipeline,sense", [(1, MAX_LE), (3, MAX_LE), (1, MIN_GE)])
def test_8192_bitwise(pipeline, sense):
    A, b, c = lpgen.dense_lp(8192, 8192, seed=0)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    g = Run(A, b, c, sense, pipeline=pipeline)
    o = oracle.solve(A, b, c, sense=sense, trace_cap=4096)
    assert g.status == o.status == capi.LP_OPTIMAL
    assert g.iters == o.iters
    assert np.array_equal(g.tp, o.trace_p) and np.array_equal(g.tq, o.trace_q)
    assert g.obj == o.obj
    assert np.array_equal(_bits(g.x), _bits(o.x)) and np.array_equal(_bits(g.y), _bits(o.y))


def test_device_pointers_and_handle_reuse():
    torch = pytest.importorskip("torch")
    h = capi.lp_create(capi.lp_options_default(trace_cap=4096))
    try:
        for (m, n) in [(300, 200), (50, 70), (400, 410)]:
            A, b, c = lpgen.dense_lp(m, n, seed=m + n)
            o = _oracle(A, b, c)
            tA, tb, tc = (torch.from_numpy(v).cuda() for v in (A, b, c))
            capi.lp_load(h, tA, tb, tc)
            capi.lp_solve(h)
            x = torch.empty(n, dtype=torch.float64, device="cuda")
            y = torch.empty(m, dtype=torch.float64, device="cuda")
            obj, st, it = capi.lp_result(h, x, y)
            assert st == capi.LP_OPTIMAL and it == o.iters and obj == o.obj
            assert np.array_equal(_bits(x.cpu().numpy()), _bits(o.x))
            assert np.array_equal(_bits(y.cpu().numpy()), _bits(o.y))
    finally:
        capi.lp_destroy(h)


def test_input_errors():
    h = capi.lp_create()
    try:
        with pytest.raises(capi.LpError) as e:
            capi.lp_solve(h)
        assert e.value.code == capi.LP_ERR_STATE
        A, b, c = lpgen.dense_lp(4, 3)
        bad = b.copy()
        bad[1] = -1.0
        capi.lp_load(h, A, bad, c)  # b < 0: taken, with Phase I (FP64)
        badc = c.copy()
        badc[0] = -2.0
        with pytest.raises(capi.LpError) as e:
            capi.lp_load(h, A, b, badc, MIN_GE)
        assert e.value.code == capi.LP_ERR_INFEASIBLE_START
        nanA = A.copy()
        nanA[2, 1] = np.nan
        with pytest.raises(capi.LpError) as e:
            capi.lp_load(h, nanA, b, c)
        assert e.value.code == capi.LP_ERR_INVALID_ARG
        # the handle still works after the rejected loads
        capi.lp_load(h, A, b, c)
        capi.lp_solve(h)
        obj, st, _ = capi.lp_result(h)
        assert st == capi.LP_OPTIMAL and obj == oracle.solve(A, b, c).obj
    finally:
        capi.lp_destroy(h)


def test_bounded_wait_times_out_and_context_survives():
    """A barrier wait limited to one cycle runs out: the kernel returns
    LP_TIMEOUT instead of hanging, and the same process solves correctly
    afterwards."""
    A, b, c = lpgen.dense_lp(600, 700, seed=1)
    o = oracle.solve(A, b, c)
    seen = set()
    for _ in range(5):
        g = Run(A, b, c, spin_timeout_cycles=1, ctas=64, threads=256)
        seen.add(g.status)
        assert g.status in (capi.LP_TIMEOUT, capi.LP_OPTIMAL)
        if g.status == capi.LP_OPTIMAL:
            assert g.obj == o.obj
    assert capi.LP_TIMEOUT in seen
    g = Run(A, b, c)
    assert g.status == capi.LP_OPTIMAL and g.obj == o.obj


_PAPER_ORACLE = {}


def _paper_case(m, n, sense, seed=1):
    """An LP of the paper's own random family and its oracle run (cached: the
    pivot-mode cases share them)."""
    A, b, c = lpgen.paper_lp(m, n, seed=seed)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    key = (m, n, sense, seed)
    if key not in _PAPER_ORACLE:
        _PAPER_ORACLE[key] = _oracle(A, b, c, sense)
    return A, b, c, _PAPER_ORACLE[key]


@pytest.mark.parametrize("pipeline", [1, 2, 4, 5])
@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
@pytest.mark.parametrize("m,n", [(40, 61), (257, 100), (100, 300), (512, 512), (1024, 1024)])
def test_paper_family_bitwise(m, n, sense, pipeline):
    """LPs of the paper's own random family (density 0.9, real-valued data;
    1445 pivots at 1024^2, against 40 for the integer family): every pivot and
    every bit as the oracle, in each primal kernel mode."""
    A, b, c, o = _paper_case(m, n, sense)
    assert o.status == oracle.OPTIMAL
    assert_same(Run(A, b, c, sense, pipeline=pipeline), o)


@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
def test_paper_family_2048_bitwise(sense):
    """2048^2 of the paper's family (2172 pivots), default launch."""
    A, b, c, o = _paper_case(2048, 2048, sense)
    assert o.status == oracle.OPTIMAL and o.iters > 2000
    assert_same(Run(A, b, c, sense), o)


@pytest.mark.parametrize("negzero", [False, True])
@pytest.mark.parametrize("pipeline", [1, 4, 5])
def test_zero_pivot_rows_and_signed_zeros(negzero, pipeline):
    """A sparse primal LP (half of A zero, so pivot rows have long zero runs),
    with its zeros stored as +0 or, in a second run, as -0 (the update turns
    some -0 entries into +0, fma(-c, +0, -0) = +0 for c < 0): every pivot and
    bit as the oracle, signed zeros included."""
    rng = np.random.default_rng(31)
    m, n = 700, 900
    A = rng.integers(1, 100, size=(m, n)).astype(np.float64)
    A[rng.random((m, n)) < 0.5] = -0.0 if negzero else 0.0
    for j in range(n):
        if not np.any(A[:, j] > 0):
            A[rng.integers(0, m), j] = 1.0
    b = rng.integers(100, 10000, size=m).astype(np.float64)
    c = rng.integers(1, 50, size=n).astype(np.float64)
    o = _oracle(A, b, c)
    assert o.status == oracle.OPTIMAL
    assert_same(Run(A, b, c, pipeline=pipeline), o)
