"""GPU parity on LPs whose rows and columns are scaled by powers of two far
from 1 (2^+-70, 2^+-130 in FP64; 2^+-90 in FP32 mode).

Scaling by powers of two keeps the data exact and leaves the LP's optimum
unchanged (row scaling does not change the feasible set; column scaling
substitutes x_j = 2^s_j x'_j).  Ratio-test operands then lie outside the
window 2^+-60 in which the screening key divides truncated single-precision
operands, so near-minimal rows mix screened and exactly divided keys in one
reduction (Sec. 2 Step 3), and FP32 tableau values approach the FP32 range.
The tolerances are set from the smallest scale so that every row and column
takes part.  FP64: every pivot and bit as the oracle in each kernel mode, and
the optimum of the unscaled LP.  FP32: the FP64 oracle's objective within
1e-6 and an FP64 certificate.
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


def scaled_lp(m, n, e, seed, rows=True, cols=True):
    """dense_lp(m, n) with row i scaled by 2^r_i and column j by 2^s_j,
    r_i, s_j drawn from {-e, 0, e}; returns the scaled LP, its tolerances
    (1e-9 times the smallest scale of each quantity) and the unscaled LP."""
    A, b, c = lpgen.dense_lp(m, n, seed=seed)
    rng = np.random.default_rng(seed + 7)
    r = rng.choice([-e, 0, e], size=m) if rows else np.zeros(m, dtype=int)
    s = rng.choice([-e, 0, e], size=n) if cols else np.zeros(n, dtype=int)
    As = np.ldexp(A, r[:, None] + s[None, :])
    bs = np.ldexp(b, r)
    cs = np.ldexp(c, s)
    lo_a = float(np.min(np.abs(As)))
    eps = dict(eps_p=1e-9 * lo_a, eps_d=1e-9 * float(np.min(np.abs(cs))),
               eps_r=1e-9 * float(np.min(np.abs(bs))))
    return (As, bs, cs), eps, (A, b, c)


@pytest.mark.parametrize("pipeline", [1, 4, 5])
@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
@pytest.mark.parametrize("e", [70, 130])
def test_scaled_bitwise(e, sense, pipeline):
    (A, b, c), eps, (A0, b0, c0) = scaled_lp(120, 150, e, seed=e + sense)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
        eps = dict(eps_p=eps["eps_p"], eps_d=eps["eps_r"], eps_r=eps["eps_d"])
    o = _oracle(A, b, c, sense, **eps)
    assert o.status == oracle.OPTIMAL
    # the optimum of the unscaled LP (the dual form: the same value by duality)
    z0 = oracle.solve(A0, b0, c0).obj
    assert abs(o.obj - z0) <= 1e-9 * abs(z0), (o.obj, z0)
    assert_same(Run(A, b, c, sense, pipeline=pipeline, **eps), o)


@pytest.mark.parametrize("reinv_k", [7, 50])
@pytest.mark.parametrize("sense", [MAX_LE, MIN_GE])
@pytest.mark.parametrize("e", [40, 56, 90])
def test_scaled_fp32_objective(e, sense, reinv_k):
    """Rows scaled by 2^+-e.  The tableau's slack columns hold entries of
    B^-1 up to about 2^(2e) in magnitude: at 2^+-40 and 2^+-56 they fit FP32
    (below 2^128) and the FP32 mode ends at the FP64 optimum (objective within
    1e-6 after the final reinversion, FP64 certificate); at 2^+-90 they do
    not, and the mode must not report a wrong optimum: it ends in
    LP_NUMERICAL or at the optimum."""
    (A, b, c), eps, (A0, b0, c0) = scaled_lp(200, 260, e, seed=11 + sense, cols=False)
    if sense == MIN_GE:
        A, b, c = lpgen.dual_of(A, b, c)
        eps = dict(eps_p=eps["eps_p"], eps_d=eps["eps_r"], eps_r=eps["eps_d"])
    o = oracle.solve(A, b, c, sense=sense, **eps)
    assert o.status == oracle.OPTIMAL
    m, n = A.shape
    h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=reinv_k,
                                               **eps))
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        x, y = np.empty(n), np.empty(m)
        obj, st, it = capi.lp_result(h, x, y)
    finally:
        capi.lp_destroy(h)
    if e >= 64:
        assert st in (capi.LP_OPTIMAL, capi.LP_NUMERICAL)
        if st == capi.LP_NUMERICAL:
            return
    assert st == capi.LP_OPTIMAL
    assert abs(obj - o.obj) <= 1e-6 * abs(o.obj), (obj, o.obj)
    cert = oracle.certificate(A, b, c, x, y, obj, sense=sense)
    # each residual against the scale of the quantities it mixes
    assert cert["gap"] <= 1e-9 * abs(o.obj) and cert["obj_vs_cx"] <= 1e-9 * abs(o.obj)
    assert cert["x_neg"] == 0.0 and cert["y_neg"] == 0.0
