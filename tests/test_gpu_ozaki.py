"""GPU: the emulated-FP64 product on the tensor cores (lp_dgemm_emulated) and
the FP32 mode's body refresh built on it.

* Integer matrices whose products and sums are exact in FP64 (entries below
  2^10, so each row and column needs two of the seven 7-bit digits): the
  product equals numpy's FP64 product bit for bit, for ragged sizes and for
  K above the 448-term chunk of an exact FP32 group sum.
* Real matrices with rows and columns scaled over six orders of magnitude:
  every entry within 2^-44 K max|A_i.| max|B_.j| of numpy's FP64 product (the
  digits keep 49 bits of each row and column scale).
* The body refresh: an FP32 solve stopped at an intermediate basis holds the
  tableau B^-1 [A I b] of that basis (oracle.reinvert, the plain definition)
  correctly rounded to FP32, in every column.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _emulated(A, B):
    tA = torch.from_numpy(np.ascontiguousarray(A)).cuda()
    tB = torch.from_numpy(np.ascontiguousarray(B)).cuda()
    tC = torch.full((A.shape[0], B.shape[1]), np.nan, dtype=torch.float64, device="cuda")
    capi.lp_dgemm_emulated(tA, tB, tC)
    return tC.cpu().numpy()


SHAPES = [(1, 1, 1), (5, 3, 7), (128, 64, 64), (130, 70, 65), (257, 300, 448), (300, 129, 449),
          (64, 200, 1000), (1000, 333, 100)]


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_integer_product_is_exact(M, N, K):
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    C = _emulated(A, B)
    assert np.array_equal(C, A @ B)


@pytest.mark.parametrize("M,N,K", SHAPES)
def test_real_product_within_the_digit_bound(M, N, K):
    rng = np.random.default_rng(M + 11 * N + 13 * K)
    A = rng.standard_normal((M, K)) * 10.0 ** rng.uniform(-3, 3, size=(M, 1))
    B = rng.standard_normal((K, N)) * 10.0 ** rng.uniform(-3, 3, size=(1, N))
    C = _emulated(A, B)
    ref = A @ B
    bound = 2.0 ** -44 * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.all(np.abs(C - ref) <= bound)


@pytest.mark.parametrize("e", [20, 60, 200])
def test_inner_scales_balanced(e):
    """A = A0 D^-1 and B = D B0 for integer A0, B0 and D = diag(2^r_k),
    r_k in {-e, 0, e}: the terms of each sum keep their magnitudes while the
    rows of A and the columns of B span 2^(2e); the inner balancing makes the
    product exact again (A B = A0 B0)."""
    rng = np.random.default_rng(e)
    M, N, K = 150, 90, 300
    A0 = rng.integers(-1000, 1001, size=(M, K)).astype(np.float64)
    B0 = rng.integers(-1000, 1001, size=(K, N)).astype(np.float64)
    r = rng.choice([-e, 0, e], size=K)
    A = np.ldexp(A0, -r[None, :])
    B = np.ldexp(B0, r[:, None])
    assert np.array_equal(_emulated(A, B), A0 @ B0)


def test_zero_rows_and_columns():
    A = np.zeros((200, 100))
    A[::3] = 1.5
    B = np.zeros((100, 90))
    B[:, ::2] = -0.25
    assert np.array_equal(_emulated(A, B), A @ B)


def _fp32_stopped(A, b, c, sense, k):
    m, n = A.shape
    h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, max_iters=k,
                                               reinv_k=10 ** 6))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        _, st, it = capi.lp_result(h)
        basis = capi.lp_get_basis(h, m)
        T = capi.lp_get_tableau(h, m, n)
        nre, _, body_ms = capi.lp_fp32_stats(h)
    finally:
        capi.lp_destroy(h)
    return st, it, basis, T, nre, body_ms


@pytest.mark.parametrize("sense", [capi.LP_MAX_LE, capi.LP_MIN_GE])
@pytest.mark.parametrize("family,m,n", [("dense", 120, 150), ("paper", 300, 420), ("paper", 700, 600)])
def test_body_refresh_matches_definition(family, m, n, sense):
    gen = lpgen.dense_lp if family == "dense" else lpgen.paper_lp
    A, b, c = gen(m, n, seed=5)
    if sense == capi.LP_MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    mm, nn = A.shape
    # the FP32 pivot sequence is its own: stop inside this run's pivots
    st, total, *_ = _fp32_stopped(A, b, c, sense, 10 ** 9)
    assert st == capi.LP_OPTIMAL and total >= 2
    for k in sorted({max(1, total // 3), total - 1}):
        st, it, basis, T, nre, body_ms = _fp32_stopped(A, b, c, sense, k)
        assert st == capi.LP_ITER_LIMIT and it == k and nre >= 1 and body_ms > 0.0
        R = oracle.reinvert(A, b, c, basis, sense=sense)
        body = T[:mm, :-1]
        want = R[:mm, :-1].astype(np.float32).astype(np.float64)
        # one FP32 rounding of the FP64 definition, plus its own FP64 error
        # (relative to the row's scale)
        ulp = np.spacing(np.abs(want).astype(np.float32)).astype(np.float64)
        tol = ulp + 1e-10 * np.abs(R[:mm, :-1]).max(axis=1, keepdims=True)
        assert np.all(np.abs(body - want) <= tol), (k, float(np.max(np.abs(body - want) - tol)))
        # basic columns are exact unit vectors
        for i, v in enumerate(basis):
            col = T[:mm, v]
            assert col[i] == 1.0 and np.count_nonzero(col) == 1


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_ill_conditioned_family_needs_the_body_refresh(seed):
    """Rows in groups of four that differ by relative 1e-4 (bases with
    condition numbers near 1e4): FP32 pivoting whose body is never refreshed
    drifts until the FP64 checks give up (LP_NUMERICAL, or an objective off by
    more than 1e-6); with the body recomputed at every reinversion the FP32
    mode ends at the FP64 oracle's optimum within 1e-6, with an FP64
    certificate."""
    A, b, c = lpgen.nearly_dependent_lp(400, 600, eps=1e-4, seed=seed)
    o = oracle.solve(A, b, c)
    assert o.status == oracle.OPTIMAL
    m, n = A.shape
    out = {}
    for body in (0, 1):
        h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50,
                                                   reinv_body=body))
        try:
            capi.lp_load(h, A, b, c)
            capi.lp_solve(h)
            x, y = np.empty(n), np.empty(m)
            obj, st, it = capi.lp_result(h, x, y)
        finally:
            capi.lp_destroy(h)
        out[body] = (st, obj, x, y)
    st0, obj0, _, _ = out[0]
    assert st0 != capi.LP_OPTIMAL or abs(obj0 - o.obj) > 1e-6 * abs(o.obj)
    st1, obj1, x1, y1 = out[1]
    assert st1 == capi.LP_OPTIMAL and abs(obj1 - o.obj) <= 1e-6 * abs(o.obj), (st1, obj1, o.obj)
    cert = oracle.certificate(A, b, c, x1, y1, obj1)
    scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
    assert max(cert.values()) <= 1e-9 * scale * 1e3, cert


def test_digit_planes_skipped_per_block():
    """Row blocks of A and column blocks of B of integer data need two of the
    seven digit planes, real-valued ones all seven; the product skips the
    planes a block does not need.  Integer block times integer block is
    exact, every entry within the digit bound."""
    rng = np.random.default_rng(77)
    M, N, K = 300, 200, 250
    A = rng.standard_normal((M, K))
    A[:128] = rng.integers(-1000, 1001, size=(128, K))   # the first row block
    B = rng.standard_normal((K, N))
    B[:, 64:128] = rng.integers(-1000, 1001, size=(K, 64))  # the second column block
    C = _emulated(A, B)
    ref = A @ B
    assert np.array_equal(C[:128, 64:128], ref[:128, 64:128])
    bound = 2.0 ** -44 * K * np.abs(A).max(axis=1)[:, None] * np.abs(B).max(axis=0)[None, :]
    assert np.all(np.abs(C - ref) <= bound)


def test_mma_count_of_the_digit_products():
    """lp_dgemm_stats: real-valued blocks need all seven digit planes, so
    every output tile runs the 28 digit pairs (p + q < 7) for every 64-deep
    K block, 4 MMAs of K = 16 each; with integer blocks (two planes) the
    product runs fewer, and never none."""
    rng = np.random.default_rng(5)
    M, N, K = 256, 128, 128  # 2 x 2 tiles of 128 x 64, 2 K blocks
    _emulated(rng.standard_normal((M, K)), rng.standard_normal((K, N)))
    assert capi.lp_dgemm_stats() == 2 * 2 * 2 * 28 * 4
    M, N, K = 300, 200, 250  # 3 x 4 tiles, 4 K blocks
    A = rng.standard_normal((M, K))
    A[:128] = rng.integers(-1000, 1001, size=(128, K))
    B = rng.standard_normal((K, N))
    B[:, 64:128] = rng.integers(-1000, 1001, size=(K, 64))
    _emulated(A, B)
    full = 3 * 4 * 4 * 28 * 4
    assert 3 * 4 * 4 * 4 <= capi.lp_dgemm_stats() < full
