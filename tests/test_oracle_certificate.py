"""Pins for the oracle's optimality certificate (no GPU).

``oracle.certificate`` is the checker behind every FP32, batch and serving
assertion, so it is pinned here on its own: each residual it reports is fed a
(x, y) pair that breaks exactly that condition by a known amount, worked out
by hand on the Wyndor worked example (tests/golden/wyndor.txt) and on its LP
dual.  The conditions are those of Eq. 1 and its dual: primal feasibility
(Ax <= b, x >= 0), dual feasibility (A'y >= c, y >= 0), equal objectives
(strong duality) and complementary slackness.  test_mutations.py plants
mistakes in copies of the function and checks that this battery fails them.
"""
import numpy as np

import oracle
from golden_io import read_lp

W = read_lp("wyndor.txt")
A, b, c = W["A"], W["b"], W["c"]  # max 3x1 + 5x2; x1 <= 4, 2x2 <= 12, 3x1 + 2x2 <= 18
XOPT, YOPT, ZOPT = W["x"], W["y"], W["z"]  # (2, 6), (0, 1.5, 1), 36

FIELDS = ("primal_infeas", "x_neg", "dual_infeas", "y_neg", "gap", "obj_vs_cx", "compl_rows",
          "compl_cols")

# (x, y, obj, expected residuals): every value below is exact in binary
# floating point, so the comparison is equality.  Each comment gives the
# hand computation.
PRIMAL_CASES = [
    # the optimum: Ax = (2, 12, 18) <= b, A'y = (3, 5) = c, c'x = b'y = 36
    ((2, 6), (0, 1.5, 1), 36, {}),
    # x2 raised by 1/4: Ax = (2, 12.5, 18.5), rows 2 and 3 over b by 0.5;
    # c'x = 37.25, so gap = obj_vs_cx = 1.25; y(b - Ax) = (0, -0.75, -0.5)
    ((2, 6.25), (0, 1.5, 1), 36,
     {"primal_infeas": 0.5, "gap": 1.25, "obj_vs_cx": 1.25, "compl_rows": 0.75}),
    # the origin, strictly feasible (Ax - b = (-4, -12, -18)): no violation,
    # gap 36, y(b - Ax) = (0, 18, 18)
    ((0, 0), (0, 1.5, 1), 36, {"gap": 36.0, "obj_vs_cx": 36.0, "compl_rows": 18.0}),
    # y3 lowered by 1/4: A'y = (2.25, 4.5), c - A'y = (0.75, 0.5);
    # b'y = 31.5, gap 4.5; x(A'y - c) = (-1.5, -3)
    ((2, 6), (0, 1.5, 0.75), 36, {"dual_infeas": 0.75, "gap": 4.5, "compl_cols": 3.0}),
    # x1 = -1: x_neg 1; Ax = (-1, 12, 9), b - Ax = (5, 0, 9), y(b - Ax) =
    # (0, 0, 9); c'x = 27, gap 9, |obj - c'x| = 9
    ((-1, 6), (0, 1.5, 1), 36, {"x_neg": 1.0, "gap": 9.0, "obj_vs_cx": 9.0, "compl_rows": 9.0}),
    # y1 = -1/2: y_neg 0.5; A'y = (2.5, 5), c - A'y = (0.5, 0); b'y = 34,
    # gap 2; y(b - Ax) = (-1, 0, 0); x(A'y - c) = (-1, 0)
    ((2, 6), (-0.5, 1.5, 1), 36,
     {"y_neg": 0.5, "dual_infeas": 0.5, "gap": 2.0, "compl_rows": 1.0, "compl_cols": 1.0}),
    # the optimum with a wrong reported objective
    ((2, 6), (0, 1.5, 1), 35, {"obj_vs_cx": 1.0}),
    # y3 = 2: A'y = (6, 7) >= c, x(A'y - c) = (6, 12); b'y = 54, gap 18
    ((2, 6), (0, 1.5, 2), 36, {"gap": 18.0, "compl_cols": 12.0}),
]

# The dual form (min c'x, Ax >= b) on Wyndor's LP dual: A_d = A', b_d = c,
# c_d = b; its optimum is x_d = y* = (0, 1.5, 1), y_d = x* = (2, 6), 36.
AD, BD, CD = A.T, c, b
DUAL_CASES = [
    ((0, 1.5, 1), (2, 6), 36, {}),
    # x_d3 lowered by 1/4: A_d x = (2.25, 4.5), b_d - A_d x = (0.75, 0.5);
    # c_d'x = 31.5, gap 4.5, obj_vs_cx 4.5; y(b - Ax) = (1.5, 3)
    ((0, 1.5, 0.75), (2, 6), 36,
     {"primal_infeas": 0.75, "gap": 4.5, "obj_vs_cx": 4.5, "compl_rows": 3.0}),
    # y_d2 raised by 1/4: A_d'y = (2, 12.5, 18.5), A_d'y - c_d = (-2, 0.5,
    # 0.5); b_d'y = 37.25, gap 1.25; x(A'y - c) = (0, 0.75, 0.5)
    ((0, 1.5, 1), (2, 6.25), 36, {"dual_infeas": 0.5, "gap": 1.25, "compl_cols": 0.75}),
    # x_d1 = -1: A_d x = (2, 5), b_d - A_d x = (1, 0), y(b - Ax) = (2, 0);
    # c_d'x = 32, gap 4; A_d'y - c_d = (-2, 0, 0), x(A'y - c) = (2, 0, 0)
    ((-1, 1.5, 1), (2, 6), 36,
     {"x_neg": 1.0, "primal_infeas": 1.0, "gap": 4.0, "obj_vs_cx": 4.0, "compl_rows": 2.0,
      "compl_cols": 2.0}),
]


def certificate_pins(cert):
    """Run every hand-computed case through `cert`; raise AssertionError on
    the first residual that differs from its expected value."""
    for cases, args, sense in ((PRIMAL_CASES, (A, b, c), oracle.MAX_LE),
                               (DUAL_CASES, (AD, BD, CD), oracle.MIN_GE)):
        for x, y, obj, want in cases:
            got = cert(*args, np.array(x, dtype=float), np.array(y, dtype=float), float(obj),
                       sense=sense)
            assert set(got) == set(FIELDS), sorted(got)
            for f in FIELDS:
                assert got[f] == want.get(f, 0.0), (sense, x, y, obj, f, got[f], want.get(f, 0.0))


def test_certificate_known_pairs():
    certificate_pins(oracle.certificate)


def test_certificate_every_field_has_a_failing_input():
    """Each residual is nonzero on at least one case of each form it applies to."""
    for cases in (PRIMAL_CASES, DUAL_CASES):
        hit = {f for _, _, _, want in cases for f in want}
        assert hit >= {"primal_infeas", "x_neg", "gap", "obj_vs_cx", "compl_rows",
                       "compl_cols", "dual_infeas"}
    assert {f for _, _, _, w in PRIMAL_CASES for f in w} == set(FIELDS)


def test_certificate_scales_with_the_violation():
    """A violation of delta along a row is reported as delta, for any delta
    (the residual is the violation itself, not a flag)."""
    for delta in (1e-12, 1e-6, 0.125, 3.0):
        got = oracle.certificate(A, b, c, np.array([2.0, 6.0 + delta / 2]), YOPT, ZOPT)
        assert abs(got["primal_infeas"] - delta) <= 1e-15 * 18
