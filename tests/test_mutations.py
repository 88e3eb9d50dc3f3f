"""Planted mistakes in the oracle: every one must fail at least one pin.

Each case copies ``oracle/simplex_oracle.c``, makes one plausible mistake (a
dropped term, a wrong sign, a wrong index, a wrong comparison), compiles the
copy with the same flags, swaps it in for the real library and runs a compact
battery of the oracle's pins.  A mutant that passes the whole battery would
mean the pins cannot tell that mistake from the correct code.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
from golden_io import read_lp
from paper_1804_04737_gb300 import lpgen

SRC = os.path.join(os.path.dirname(oracle.__file__), "simplex_oracle.c")
CAP = 5000

MUTANTS = {
    "update_sign": ("const double a = -col[i];", "const double a = col[i];"),
    "pricing_max": ("if (q < 0 || z[j] < best)", "if (q < 0 || z[j] > best)"),
    "no_row_division": ("prow[j] = rowp[j] / piv;", "prow[j] = rowp[j];"),
    "ratio_max": ("if (p < 0 || r < best ||", "if (p < 0 || r > best ||"),
    "objective_row_skipped": ("for (int i = 0; i < M; ++i) {\n        if (i == p) continue;",
                              "for (int i = 0; i < M - 1; ++i) {\n        if (i == p) continue;"),
    "rhs_column_off_by_one": ("const double rhs = T[(long)i * N + N - 1];",
                              "const double rhs = T[(long)i * N + N - 2];"),
    "no_ratio_clamp": ("const double r = (rhs > 0.0 ? rhs : 0.0) / a;",
                       "const double r = (rhs > 0.0 ? 0.0 : rhs) / a;"),
    "slack_identity_missing": ("row[n + i] = 1.0;", "row[n + i] = 2.0;"),
    "dual_values_index": ("y[i] = z[n + i];", "y[i] = z[i];"),
    "dual_leave_max": ("} else if (r < 0 || v < best) {", "} else if (r < 0 || v > best) {"),
    "dual_ratio_sign": ("const double t = zj / (-a);", "const double t = zj / a;"),
    "bland_tiebreak": ("const int key = bland ? basis[i] : i;", "const int key = i;"),
    "never_bland": ("*deg = (rmin == 0.0) ? *deg + 1 : 0;", "*deg = 0;"),
    "phase2_term_sign": ("z[j] = fma(cb, row[j], z[j]);", "z[j] = fma(-cb, row[j], z[j]);"),
    "phase2_objective_value_skipped": ("for (long j = 0; j < N; ++j) z[j] = fma(cb, row[j], z[j]);",
                                       "for (long j = 0; j < N - 1; ++j) z[j] = fma(cb, row[j], z[j]);"),
    "primal_objective_sign": ("*obj = (sense == OR_MAX_LE) ? z[N - 1] : -z[N - 1];",
                              "*obj = (sense == OR_MAX_LE) ? z[N - 1] : z[N - 1];"),
}


def _pins():
    """Compact pin battery; raises AssertionError on the first failure."""
    rel = lambda a, b: abs(a - b) / max(1.0, abs(b))  # noqa: E731
    # brute force, primal and dual forms
    for seed in range(60):
        rng = np.random.default_rng(seed)
        m, n = (int(v) for v in rng.integers(1, 6, size=2))
        A = rng.uniform(0.05, 10.0, size=(m, n))
        b = rng.uniform(0.5, 10.0, size=m)
        c = rng.uniform(-1.0, 5.0, size=n)
        r = oracle.solve(A, b, c, max_iters=CAP)
        z, _ = oracle.brute_force(A, b, c)
        assert r.status == oracle.OPTIMAL and rel(r.obj, z) <= 1e-9
        cert = oracle.certificate(A, b, c, r.x, r.y, r.obj)
        assert max(cert.values()) <= 1e-8 * max(1.0, abs(z))
        cd = np.abs(c)
        rd = oracle.solve(A, b, cd, sense=oracle.MIN_GE, max_iters=CAP)
        zd, _ = oracle.brute_force(A.T, cd, b)
        assert rd.status == oracle.OPTIMAL and rel(rd.obj, zd) <= 1e-9
        cert = oracle.certificate(A, b, cd, rd.x, rd.y, rd.obj, sense=oracle.MIN_GE)
        assert max(cert.values()) <= 1e-8 * max(1.0, abs(zd))
    # cycling examples terminate at the printed optimum with Bland's rule
    for name in ("chvatal_cycling.txt", "beale_cycling.txt"):
        g = read_lp(name)
        for ba in (0, 32):
            r = oracle.solve(g["A"], g["b"], g["c"], bland_after=ba, max_iters=CAP)
            assert r.status == oracle.OPTIMAL and rel(r.obj, g["z"]) <= 1e-12
    g = read_lp("bland_tie.txt")
    for ba, key in ((0, "bland"), (10 ** 9, "dantzig")):
        r = oracle.solve(g["A"], g["b"], g["c"], bland_after=ba, trace_cap=10, max_iters=CAP)
        got = np.stack([r.trace_p, r.trace_q], axis=1).ravel()[:len(g[key])]
        assert got.tolist() == g[key].astype(int).tolist()
    # primal and dual formulations agree, pivot for pivot count
    A, b, c = lpgen.dense_lp(40, 70, seed=5)
    rp = oracle.solve(A, b, c, max_iters=CAP)
    rd = oracle.solve(*lpgen.dual_of(A, b, c), sense=oracle.MIN_GE, max_iters=CAP)
    assert rp.status == rd.status == oracle.OPTIMAL
    assert rel(rd.obj, rp.obj) <= 1e-12 and rp.iters == rd.iters
    # Phase I (some b_i < 0): brute force on bounded LPs, a hand-solved case
    done = 0
    for seed in range(200):
        rng = np.random.default_rng(1000 + seed)
        m, n = (int(v) for v in rng.integers(2, 5, size=2))
        A = rng.integers(-4, 6, size=(m, n)).astype(float)
        b = rng.integers(-5, 12, size=m).astype(float)
        A[0] = rng.integers(1, 5, size=n)
        b[0] = abs(b[0]) + 5.0
        if not np.any(b < 0):
            continue
        c = rng.integers(-3, 6, size=n).astype(float)
        r = oracle.solve(A, b, c, max_iters=CAP)
        z, _ = oracle.brute_force(A, b, c)
        if z is None:
            assert r.status == oracle.INFEASIBLE
        else:
            assert r.status == oracle.OPTIMAL and rel(r.obj, z) <= 1e-9
            done += 1
    assert done > 30
    r = oracle.solve(np.array([[1.0, 1.0], [-1.0, -1.0], [1.0, 0.0]]), np.array([4.0, -2.0, 3.0]),
                     np.array([2.0, 3.0]), max_iters=CAP)
    assert r.status == oracle.OPTIMAL and r.obj == 12.0 and np.array_equal(r.x, [0.0, 4.0])


def _build_mutant(tmp_path, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, old
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                    "-std=c11", "-o", str(lib), str(path), "-lm"], check=True, timeout=120)
    return oracle._bind(ctypes.CDLL(str(lib)))


def test_unmutated_passes():
    _pins()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    monkeypatch.setattr(oracle, "_lib", _build_mutant(tmp_path, old, new))
    with pytest.raises(AssertionError):
        _pins()


# Planted mistakes in copies of oracle.certificate (the checker behind every
# FP32, batch and serving assertion); the hand-computed battery of
# test_oracle_certificate.py must fail each one.
CERT_MUTANTS = {
    "dropped_max": ("primal = max(0.0, float(np.max(Ax - b)) if len(b) else 0.0)",
                    "primal = float(np.max(Ax - b)) if len(b) else 0.0"),
    "dual_sign_swapped": ("dual = max(0.0, float(np.max(c - Aty)) if len(c) else 0.0)",
                          "dual = max(0.0, float(np.max(Aty - c)) if len(c) else 0.0)"),
    "min_form_primal_sign": ("primal = max(0.0, float(np.max(b - Ax)) if len(b) else 0.0)",
                             "primal = max(0.0, float(np.max(Ax - b)) if len(b) else 0.0)"),
    "x_neg_from_max": ('"x_neg": max(0.0, float(-np.min(x)) if len(x) else 0.0)',
                       '"x_neg": max(0.0, float(-np.max(x)) if len(x) else 0.0)'),
    "gap_against_obj": ('"gap": abs(float(c @ x) - float(b @ y))',
                        '"gap": abs(obj - float(b @ y))'),
    "compl_rows_self": ('np.abs(y * (b - Ax))', 'np.abs(y * (Ax - Ax))'),
    "compl_cols_transposed": ("Aty = A.T @ y", "Aty = A.T @ y[::-1]"),
}


def _mutant_certificate(old, new):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(oracle.certificate))
    assert src.count(old) == 1, old
    ns = {"np": np, "MAX_LE": oracle.MAX_LE}
    exec(compile(src.replace(old, new), "<mutant certificate>", "exec"), ns)
    return ns["certificate"]


def test_unmutated_certificate_passes():
    from test_oracle_certificate import certificate_pins
    certificate_pins(_mutant_certificate("Aty = A.T @ y", "Aty = A.T @ y"))


@pytest.mark.parametrize("name", sorted(CERT_MUTANTS))
def test_certificate_mutant_is_caught(name):
    from test_oracle_certificate import certificate_pins
    with pytest.raises(AssertionError):
        certificate_pins(_mutant_certificate(*CERT_MUTANTS[name]))
