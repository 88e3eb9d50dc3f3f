"""Seeded synthetic dense-LP generators (inputs only; no simplex arithmetic).

These stand in for the paper's random instances (Sec. 4 generates dense LPs
of sizes 256..8192 with an Octave routine whose text is garbled and whose
random stream is not reproducible here): ``dense_lp`` is the main family
(integer data, exact in FP32), ``paper_lp`` follows the paper's own
distribution.  Both the CUDA library's tests and the CPU oracle take their
inputs from this module.

Dense workload (one LP):
  A_ij  iid uniform integers in [1, 1000]     (row-major, drawn first)
  b_i   iid uniform integers in [1000, 100000] (drawn second)
  c_j   iid uniform integers in [1, 100]       (drawn third)
all from ``numpy.random.default_rng(seed)`` and stored as float64.  Every
value is an integer below 2**24, so it is exact in FP32 as well.  A > 0 and
b > 0 make the LP max c'x, Ax <= b, x >= 0 feasible (x = 0) and bounded.
"""
import numpy as np


def dense_lp(m: int, n: int, seed: int = 0):
    """(A, b, c) of one dense LP, float64, C-contiguous."""
    rng = np.random.default_rng(seed)
    A = rng.integers(1, 1001, size=(m, n)).astype(np.float64)
    b = rng.integers(1000, 100001, size=m).astype(np.float64)
    c = rng.integers(1, 101, size=n).astype(np.float64)
    return A, b, c


def paper_lp(m: int, n: int, seed: int = 0, density: float = 0.9):
    """(A, b, c) of one LP of the paper's own random family (Sec. 4), float64.

    The paper draws A with a given density (0.9 in its runs) and nonzeros
    uniform on (0, 50), a point x0 with entries uniform on [0, 10), b = A x0
    (so x0 is feasible and b >= 0), and an objective row A'u for a random
    vector u, redrawn until that row has a negative entry.  The listing that
    states this is garbled (its objective assignment reads "c=A'"); the reading
    taken here is objective row = A'u with u_i = [r1 > r2] (r3 - r4) for
    uniform r's, as its other lines define u.  In the form max c'x, Ax <= b
    used here the objective row is -c, so c = -A'u.

    Draw order (``numpy.random.default_rng(seed)``), repeated until c has a
    positive entry: A's values, A's mask, x0, then r1, r2, r3, r4 (m each).
    Unlike ``dense_lp`` the values are not integers: FP32 holds them rounded."""
    rng = np.random.default_rng(seed)
    while True:
        vals = 50.0 * rng.random((m, n))
        mask = rng.random((m, n)) < density
        A = np.where(mask, vals, 0.0)
        x0 = 10.0 * rng.random(n)
        b = A @ x0
        r1, r2, r3, r4 = (rng.random(m) for _ in range(4))
        u = np.where(r1 > r2, r3 - r4, 0.0)
        c = -(A.T @ u)
        if np.any(c > 0):
            return (np.ascontiguousarray(A), np.ascontiguousarray(b), np.ascontiguousarray(c))


def nearly_dependent_lp(m: int, n: int, eps: float = 1e-4, seed: int = 0, group: int = 4):
    """(A, b, c) of an ill-conditioned dense LP: its rows come in groups of
    `group` that are relative perturbations of size `eps` of one common row,
    so bases holding several rows of a group have condition numbers near
    1 / eps.  Feasible and bounded: A > 0 (for eps well below 1), c > 0, and
    b = A x0 + a small positive slack for x0 >= 0.

    Draw order (``numpy.random.default_rng(seed)``): the common rows (uniform
    on [1, 100)), the perturbations (standard normal), x0 (uniform on
    [0, 1)), the slack (uniform on [0, 0.01)), c (uniform on [1, 100))."""
    rng = np.random.default_rng(seed)
    base = rng.uniform(1.0, 100.0, size=(m // group + 1, n))
    A = base[np.arange(m) // group] * (1.0 + eps * rng.standard_normal((m, n)))
    b = A @ rng.uniform(0.0, 1.0, size=n) + rng.uniform(0.0, 1e-2, size=m)
    c = rng.uniform(1.0, 100.0, size=n)
    return (np.ascontiguousarray(A), np.ascontiguousarray(b), np.ascontiguousarray(c))


def with_ge_rows(A, b, frac: float = 0.1, seed: int = 0):
    """(A', b') with a fraction of the rows of a positive LP turned into >=
    rows that the origin violates, so that the primal form needs Phase I.

    With x0 = t * 1 for t = min_i b_i / sum_j A_ij / 2 (so A x0 <= b / 2 on
    every row), each chosen row i (``numpy.random.default_rng(seed)``,
    without replacement) becomes a_i x >= a_i x0 / 2, stored as
    -a_i x <= -(a_i x0) / 2.  x0 satisfies every row, so the LP is feasible,
    and the rows left as <= rows keep it bounded when A > 0."""
    A = np.array(A, dtype=np.float64, copy=True)
    b = np.array(b, dtype=np.float64, copy=True)
    m = A.shape[0]
    rs = A.sum(axis=1)
    t = 0.5 * float(np.min(b / rs))
    k = max(1, int(round(frac * m)))
    rows = np.random.default_rng(seed).choice(m, size=min(k, m), replace=False)
    b[rows] = -0.5 * t * rs[rows]
    A[rows] = -A[rows]
    return A, b


def dual_of(A, b, c):
    """Data of the dual LP  min b'y  s.t.  A'y >= c, y >= 0  as (A', c, b).

    Feed the result to the dual-form entry point (min c'x, Ax >= b)."""
    return np.ascontiguousarray(np.asarray(A).T), np.asarray(c).copy(), np.asarray(b).copy()


def log_uniform_shapes(count: int, lo: int, hi: int, seed: int = 0):
    """`count` (m, n) pairs, each drawn log-uniformly in [lo, hi] (integers)."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(np.log(lo), np.log(hi), size=(count, 2))
    s = np.clip(np.rint(np.exp(u)).astype(np.int64), lo, hi)
    return [(int(a), int(b)) for a, b in s]


def batch_lps(count: int, lo: int, hi: int, seed: int = 0):
    """`count` dense LPs with log-uniform shapes; LP k uses seed (seed, k)."""
    shapes = log_uniform_shapes(count, lo, hi, seed)
    out = []
    for k, (m, n) in enumerate(shapes):
        out.append(dense_lp(m, n, seed=np.random.SeedSequence([seed, k]).generate_state(1)[0]))
    return out


def poisson_arrivals(count: int, rate_per_s: float, seed: int = 0):
    """Arrival times (seconds from 0) of a Poisson stream with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
