"""Pins for the FP64 CPU oracle (no GPU).

The oracle is checked against things fixed independently of it: brute-force
vertex enumeration, literature examples with printed optima and pivot counts,
LP duality, a library LP solver, and the direct B^-1 definition of the
tableau.  Planted mistakes (test_mutations.py) show each pin has teeth.
"""
import numpy as np
import pytest

import oracle
from golden_io import read_lp, read_table
from paper_1804_04737_gb300 import lpgen

CERT_TOL = 1e-9


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


def _random_small(seed, integer=False):
    rng = np.random.default_rng(seed)
    m, n = (int(v) for v in rng.integers(1, 7, size=2))
    if integer:
        A = rng.integers(0, 4, size=(m, n)).astype(float)
        b = rng.integers(0, 6, size=m).astype(float)
        c = rng.integers(-2, 5, size=n).astype(float)
        # A >= 0 and every column has a positive entry: the LP is bounded
        for j in range(n):
            if not np.any(A[:, j] > 0):
                A[rng.integers(0, m), j] = 1.0 + rng.integers(0, 3)
    else:
        A = rng.uniform(0.05, 10.0, size=(m, n))
        b = rng.uniform(0.5, 10.0, size=m)
        c = rng.uniform(-1.0, 5.0, size=n)
    return A, b, c


@pytest.mark.parametrize("integer", [False, True])
def test_brute_force_small(integer):
    """Eq. 1 optimum by vertex enumeration, m, n <= 6 (integer data forces ties
    and degenerate vertices)."""
    for seed in range(250):
        A, b, c = _random_small(seed, integer)
        r = oracle.solve(A, b, c)
        z, _ = oracle.brute_force(A, b, c)
        assert r.status == oracle.OPTIMAL, seed
        assert _rel(r.obj, z) <= 1e-9, (seed, r.obj, z)
        cert = oracle.certificate(A, b, c, r.x, r.y, r.obj)
        assert max(cert.values()) <= 1e-8 * max(1.0, abs(z)), (seed, cert)


def test_brute_force_dual_form():
    """min c'x, Ax >= b by the dual simplex equals the brute-force optimum of
    its LP dual max b'y, A'y <= c (strong duality)."""
    for seed in range(200):
        rng = np.random.default_rng(1000 + seed)
        m, n = (int(v) for v in rng.integers(1, 7, size=2))
        A = rng.uniform(0.05, 10.0, size=(m, n))
        b = rng.uniform(-2.0, 10.0, size=m)
        c = rng.uniform(0.0, 5.0, size=n)
        r = oracle.solve(A, b, c, sense=oracle.MIN_GE)
        # dual of min c'x, Ax >= b, x >= 0 is max b'y, A'y <= c, y >= 0
        z, _ = oracle.brute_force(A.T, c, b)
        assert r.status == oracle.OPTIMAL, seed
        assert _rel(r.obj, z) <= 1e-9, (seed, r.obj, z)
        cert = oracle.certificate(A, b, c, r.x, r.y, r.obj, sense=oracle.MIN_GE)
        assert max(cert.values()) <= 1e-8 * max(1.0, abs(z)), (seed, cert)


def test_wyndor_textbook():
    g = read_lp("wyndor.txt")
    r = oracle.solve(g["A"], g["b"], g["c"])
    assert r.status == oracle.OPTIMAL
    assert r.obj == g["z"]
    np.testing.assert_allclose(r.x, g["x"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(r.y, g["y"], rtol=0, atol=1e-12)


def test_klee_minty_pivot_counts():
    """Dantzig's rule takes 2^n - 1 pivots on the Klee-Minty cube (golden)."""
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
        r = oracle.solve(A, b, c, trace_cap=1 << 10)
        assert r.status == oracle.OPTIMAL
        assert r.iters == int(pivots)
        assert r.obj == z
        # the iteration cap stops it exactly there, and the run resumes
        t = oracle.OracleTableau(A, b, c)
        assert t.run(max_iters=int(pivots) // 2) == oracle.ITER_LIMIT
        assert t.iters.value == int(pivots) // 2
        assert t.run() == oracle.OPTIMAL and t.iters.value == int(pivots)


@pytest.mark.parametrize("name", ["chvatal_cycling.txt", "beale_cycling.txt"])
def test_cycling_examples(name):
    """Pure Dantzig cycles with the printed period; the Bland fallback ends at
    the printed optimum."""
    g = read_lp(name)
    A, b, c = g["A"], g["b"], g["c"]
    r = oracle.solve(A, b, c, bland_after=10 ** 9, max_iters=60, trace_cap=60)
    assert r.status == oracle.ITER_LIMIT
    k = int(g["cycle"])
    assert np.array_equal(r.trace_p[:k], r.trace_p[k:2 * k])
    assert np.array_equal(r.trace_q[:k], r.trace_q[k:2 * k])
    for ba in (0, 1, 32):
        r = oracle.solve(A, b, c, bland_after=ba)
        assert r.status == oracle.OPTIMAL
        assert _rel(r.obj, g["z"]) <= 1e-12
    assert _rel(oracle.brute_force(A, b, c)[0], g["z"]) <= 1e-12


def test_bland_leaving_tiebreak():
    """Hand-derived traces: Bland's rule breaks a ratio tie by the smallest
    basic-variable index, Dantzig mode by the smallest row (golden)."""
    g = read_lp("bland_tie.txt")
    for ba, key in ((0, "bland"), (10 ** 9, "dantzig")):
        r = oracle.solve(g["A"], g["b"], g["c"], bland_after=ba, trace_cap=10)
        assert r.status == oracle.OPTIMAL and r.obj == g["z"]
        exp = g[key].astype(int)
        got = np.stack([r.trace_p, r.trace_q], axis=1).ravel()[:len(exp)]
        assert got.tolist() == exp.tolist()


def test_diagonal_closed_form():
    """A = diag(a): z* = sum c_i b_i / a_i, n pivots, entering order by c
    descending (ties: smallest index), leaving row = entering index."""
    rng = np.random.default_rng(7)
    n = 40
    a = rng.integers(1, 20, size=n).astype(float)
    b = rng.integers(1, 50, size=n).astype(float)
    c = rng.integers(1, 10, size=n).astype(float)
    r = oracle.solve(np.diag(a), b, c, trace_cap=n)
    assert r.status == oracle.OPTIMAL and r.iters == n
    order = sorted(range(n), key=lambda j: (-c[j], j))
    assert list(r.trace_q) == order
    assert list(r.trace_p) == order
    assert _rel(r.obj, float(np.sum(c * b / a))) <= 1e-14


def test_single_constraint_closed_form():
    rng = np.random.default_rng(8)
    for _ in range(50):
        n = int(rng.integers(1, 30))
        a = rng.uniform(0.5, 5.0, size=n)
        c = rng.uniform(0.1, 3.0, size=n)
        b = float(rng.uniform(1.0, 10.0))
        r = oracle.solve(a[None, :], np.array([b]), c)
        assert r.status == oracle.OPTIMAL
        assert _rel(r.obj, b * float(np.max(c / a))) <= 1e-13


def test_unbounded():
    """Step 3: a candidate column with no positive entry => unbounded."""
    A = np.array([[1.0, -1.0], [2.0, 0.0]])
    b = np.array([4.0, 6.0])
    c = np.array([1.0, 3.0])
    r = oracle.solve(A, b, c)
    assert r.status == oracle.UNBOUNDED and r.iters == 0
    # unbounded after one pivot
    A = np.array([[1.0, -1.0]])
    r = oracle.solve(A, np.array([2.0]), np.array([2.0, 1.0]))
    assert r.status == oracle.UNBOUNDED and r.iters == 1


def test_dual_form_infeasible():
    """Dual simplex: a violated row with no negative entry => infeasible."""
    A = np.array([[-1.0, -2.0]])  # -x1 - 2 x2 >= 1 has no x >= 0
    r = oracle.solve(A, np.array([1.0]), np.array([1.0, 1.0]), sense=oracle.MIN_GE)
    assert r.status == oracle.INFEASIBLE


def test_zero_and_trivial_sizes():
    # c <= 0: slack basis optimal, no pivots
    r = oracle.solve(np.ones((3, 2)), np.ones(3), -np.ones(2))
    assert r.status == oracle.OPTIMAL and r.iters == 0 and r.obj == 0.0
    # b = 0: degenerate from the start, optimum 0
    r = oracle.solve(np.ones((3, 2)), np.zeros(3), np.ones(2))
    assert r.status == oracle.OPTIMAL and r.obj == 0.0
    # 1 x 1
    r = oracle.solve(np.array([[4.0]]), np.array([2.0]), np.array([3.0]))
    assert r.status == oracle.OPTIMAL and r.obj == 1.5 and r.iters == 1


@pytest.mark.parametrize("gen", ["dense_lp", "paper_lp"])
@pytest.mark.parametrize("m,n", [(64, 64), (96, 200), (200, 96)])
def test_generator_instances_certificate_and_linprog(m, n, gen):
    """Generator LPs (both families): optimality certificate, and the optimum
    of a library LP solver (HiGHS via scipy)."""
    A, b, c = getattr(lpgen, gen)(m, n, seed=3)
    r = oracle.solve(A, b, c)
    assert r.status == oracle.OPTIMAL
    cert = oracle.certificate(A, b, c, r.x, r.y, r.obj)
    scale = max(1.0, abs(r.obj), float(np.max(b)))
    assert max(cert.values()) <= 1e-12 * scale * 1e3, cert
    sp = pytest.importorskip("scipy.optimize")
    res = sp.linprog(-c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
    assert res.status == 0
    assert _rel(r.obj, -res.fun) <= 1e-9


@pytest.mark.parametrize("gen", ["dense_lp", "paper_lp"])
@pytest.mark.parametrize("m,n", [(64, 64), (50, 120), (120, 50)])
def test_dual_form_matches_primal(m, n, gen):
    """Sec. 4 solves each problem in primal and dual formulation: the same
    optimum, x of one is y of the other."""
    A, b, c = getattr(lpgen, gen)(m, n, seed=5)
    rp = oracle.solve(A, b, c)
    Ad, bd, cd = lpgen.dual_of(A, b, c)
    rd = oracle.solve(Ad, bd, cd, sense=oracle.MIN_GE)
    assert rp.status == rd.status == oracle.OPTIMAL
    assert _rel(rd.obj, rp.obj) <= 1e-12
    assert rp.iters == rd.iters
    np.testing.assert_allclose(rd.x, rp.y, rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(rd.y, rp.x, rtol=1e-9, atol=1e-9)


def test_tableau_invariants_each_pivot():
    """After every pivot the basic columns are exact unit vectors (Step 5:
    pivot column becomes zero except the pivot element, which is one)."""
    A, b, c = lpgen.dense_lp(40, 60, seed=11)
    t = oracle.OracleTableau(A, b, c)
    m = 40
    for k in range(1, 200):
        st = t.run(max_iters=k)
        T = t.T
        for i, j in enumerate(t.basis):
            col = T[:, j]
            assert col[i] == 1.0
            assert np.all(col[np.arange(m + 1) != i] == 0.0)
        assert np.all(T[:m, -1] >= 0.0)  # primal feasible throughout
        if st != oracle.ITER_LIMIT:
            break
    assert st == oracle.OPTIMAL


@pytest.mark.parametrize("sense", [oracle.MAX_LE, oracle.MIN_GE])
def test_reinversion_definition_matches_pivots(sense):
    """The tableau after k pivots equals B^-1 [A I b] of its basis."""
    A, b, c = lpgen.dense_lp(30, 45, seed=2)
    if sense == oracle.MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
    t = oracle.OracleTableau(A, b, c, sense=sense)
    for k in (1, 3, 7, 100):
        t.run(max_iters=k)
        R = oracle.reinvert(A, b, c, t.basis, sense=sense)
        scale = np.maximum(1.0, np.abs(R))
        assert np.max(np.abs(t.T - R) / scale) <= 1e-9


def test_resume_and_threads_bitwise():
    A, b, c = lpgen.dense_lp(300, 257, seed=4)
    oracle.set_threads(1)
    full = oracle.solve(A, b, c, trace_cap=1000, keep_tableau=True)
    t = oracle.OracleTableau(A, b, c, trace_cap=1000)
    k = 0
    while t.run(max_iters=k) == oracle.ITER_LIMIT:
        k += 3
    step = t.result(keep_tableau=True)
    oracle.set_threads(4)
    par = oracle.solve(A, b, c, trace_cap=1000, keep_tableau=True)
    oracle.set_threads(1)
    for r in (step, par):
        assert r.iters == full.iters
        assert np.array_equal(r.trace_p, full.trace_p)
        assert np.array_equal(r.trace_q, full.trace_q)
        assert np.array_equal(r.T.view(np.uint64), full.T.view(np.uint64))


def test_input_validation():
    with pytest.raises(ValueError):
        oracle.solve(np.ones((2, 2)), np.ones(2), np.array([1.0, -1.0]), sense=oracle.MIN_GE)


def test_paper_family_generator():
    """The paper's random family (Sec. 4): density 0.9, nonzeros in (0, 50),
    b = A x0 >= 0 for some x0 >= 0 (so x0 is feasible), an objective with an
    improving column; the same seed gives the same LP."""
    A, b, c = lpgen.paper_lp(300, 400, seed=7)
    assert A.shape == (300, 400) and b.shape == (300,) and c.shape == (400,)
    assert abs(float(np.mean(A > 0)) - 0.9) < 0.01
    assert float(A.min()) >= 0.0 and float(A.max()) < 50.0
    assert np.all(b >= 0) and np.any(c > 0)
    # b lies in the cone of A's columns: a nonnegative x with A x = b exists
    sp = pytest.importorskip("scipy.optimize")
    x, res = sp.nnls(A, b)
    assert res <= 1e-9 * float(np.linalg.norm(b))
    A2, b2, c2 = lpgen.paper_lp(300, 400, seed=7)
    assert np.array_equal(A, A2) and np.array_equal(b, b2) and np.array_equal(c, c2)


# ---- Phase I (the primal form with some b_i < 0; not in the paper) ----

def _small_mixed(rng, lo=1, hi=7):
    m, n = (int(v) for v in rng.integers(lo, hi, size=2))
    A = rng.integers(-5, 6, size=(m, n)).astype(float)
    b = rng.integers(-6, 10, size=m).astype(float)
    c = rng.integers(-3, 6, size=n).astype(float)
    return A, b, c


def test_phase1_vs_highs():
    """Random small LPs with negative right-hand sides: status and optimum
    agree with HiGHS (its presolve's "infeasible or unbounded" is settled by
    a feasibility solve)."""
    sp = pytest.importorskip("scipy.optimize")
    rng = np.random.default_rng(11)
    seen = set()
    for _ in range(600):
        A, b, c = _small_mixed(rng)
        r = oracle.solve(A, b, c)
        res = sp.linprog(-c, A_ub=A, b_ub=b, bounds=(0, None), method="highs")
        if res.status not in (0, 2, 3):
            continue  # HiGHS gave no answer (numerical difficulties)
        if res.status == 2:
            feas = sp.linprog(np.zeros(len(c)), A_ub=A, b_ub=b, bounds=(0, None),
                              method="highs").status == 0
            want = oracle.UNBOUNDED if feas else oracle.INFEASIBLE
        else:
            want = {0: oracle.OPTIMAL, 3: oracle.UNBOUNDED}[res.status]
        assert r.status == want, (A, b, c, r.status, res.status)
        if want == oracle.OPTIMAL:
            assert _rel(r.obj, -res.fun) <= 1e-9
            assert np.all(A @ r.x <= b + 1e-9) and np.all(r.x >= -1e-12)
        seen.add(want)
    assert seen == {oracle.OPTIMAL, oracle.UNBOUNDED, oracle.INFEASIBLE}


def test_phase1_brute_force():
    """Bounded LPs with some b_i < 0: the optimum equals the best vertex."""
    rng = np.random.default_rng(12)
    done = 0
    for _ in range(400):
        m, n = (int(v) for v in rng.integers(2, 6, size=2))
        A = rng.integers(-4, 6, size=(m, n)).astype(float)
        b = rng.integers(-5, 12, size=m).astype(float)
        A[0] = rng.integers(1, 5, size=n)   # a row that bounds every x_j
        b[0] = abs(b[0]) + 5.0
        if not np.any(b < 0):
            continue
        c = rng.integers(-3, 6, size=n).astype(float)
        r = oracle.solve(A, b, c)
        z, _ = oracle.brute_force(A, b, c)
        if z is None:
            assert r.status == oracle.INFEASIBLE
        else:
            assert r.status == oracle.OPTIMAL and abs(r.obj - z) <= 1e-9 * max(1.0, abs(z))
            done += 1
    assert done > 100


def test_phase1_textbook():
    """max 2x1 + 3x2 s.t. x1 + x2 <= 4, x1 + x2 >= 2, x1 <= 3: the optimum is
    x = (0, 4), z = 12, and the origin is infeasible, so Phase 1 pivots first."""
    A = np.array([[1.0, 1.0], [-1.0, -1.0], [1.0, 0.0]])
    b = np.array([4.0, -2.0, 3.0])
    c = np.array([2.0, 3.0])
    r = oracle.solve(A, b, c, trace_cap=10)
    assert r.status == oracle.OPTIMAL and r.obj == 12.0
    assert np.array_equal(r.x, [0.0, 4.0])
    assert r.trace_p[0] == 1  # Phase 1 leaves the violated row first


def test_phase1_infeasible():
    """x1 + x2 <= -1 has no x >= 0: Phase 1 finds no entering column."""
    r = oracle.solve(np.array([[1.0, 1.0], [1.0, 0.0]]), np.array([-1.0, 3.0]),
                     np.array([1.0, 1.0]))
    assert r.status == oracle.INFEASIBLE and r.iters == 0


def test_phase1_resume_in_chunks():
    """Stopping every few pivots (across the switch to Phase 2) and resuming
    gives the bits of one run."""
    rng = np.random.default_rng(13)
    A = rng.integers(1, 20, size=(30, 40)).astype(float)
    b = rng.integers(50, 200, size=30).astype(float)
    A[:6] = -A[:6]
    b[:6] = -0.2 * b[:6]
    c = rng.integers(1, 30, size=40).astype(float)
    one = oracle.solve(A, b, c, trace_cap=500, keep_tableau=True)
    assert one.status == oracle.OPTIMAL and one.iters > 10
    t = oracle.OracleTableau(A, b, c, trace_cap=500)
    k = 0
    while True:
        k += 3
        if t.run(k) != oracle.ITER_LIMIT:
            break
    r = t.result(keep_tableau=True)
    assert r.status == one.status and r.iters == one.iters
    assert np.array_equal(r.trace_p, one.trace_p) and np.array_equal(r.trace_q, one.trace_q)
    assert np.array_equal(r.T.view(np.uint64), one.T.view(np.uint64))
