"""GPU: servers that spill idle LPs to host memory (lp_options.spill_pivots).

An LP that has pivoted spill_pivots times since its last admission and is
idle on the device may have its tableau and state copied to pinned host
memory and go to the back of the queue when the request at the head cannot
be admitted; readmitted, it pivots on where it stopped.  Sec. 2's iteration
is a function of the tableau and the basis alone, so a solve that is spilled
and readmitted any number of times must give every bit that one solve in one
place gives:

* FP64, LPs that run alone (solo_elems): solved in slices of spill_pivots
  pivots, spilled after a slice when requests wait; the oracle's bits, also
  at an iteration limit that falls inside a slice, and with two such LPs
  taking turns;
* FP32 rounds: spilled between rounds under a budget that holds two LPs; the
  same bits as a server with room for all of them, objective within the FP32
  mode's tolerance of the oracle.
"""
import os
import time

import numpy as np
import pytest

import oracle
from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()
    oracle.set_threads(os.cpu_count() or 1)
    yield
    oracle.set_threads(1)


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _small(count, seed):
    return [(*lpgen.dense_lp(m, n, seed=900 * seed + k), capi.LP_MAX_LE)
            for k, (m, n) in enumerate(lpgen.log_uniform_shapes(count, 10, 80, seed))]


def _same_as_oracle(lp, res, **kw):
    A, b, c, sense = lp
    obj, st, it, x, y, lat = res
    o = oracle.solve(A, b, c, sense=sense, **kw)
    assert st == o.status and it == o.iters
    assert _bits([obj])[0] == _bits([o.obj])[0]
    assert np.array_equal(_bits(x), _bits(o.x)) and np.array_equal(_bits(y), _bits(o.y))


def _run(srv, lps):
    """Submit all, then wait for all; (results, host-clock done times)."""
    sub = []
    for lp in lps:
        sub.append((capi.lp_server_submit(srv, *lp), time.perf_counter()))
    res, done = [], []
    for lp, (t, t0) in zip(lps, sub):
        r = capi.lp_server_wait(srv, t, lp[0].shape[0], lp[0].shape[1], timeout_s=300.0)
        res.append(r)
        done.append(t0 + r[5] * 1e-3)
    return res, done


@pytest.mark.parametrize("lanes", [0, 3])
def test_fp64_large_lp_sliced_and_spilled(lanes):
    """A large LP (alone, in slices of 40 pivots) submitted just before 24
    small ones: it is spilled while they wait, they finish before it, and
    every result is the oracle's, bit for bit; with the server kernel or
    with three lanes serving the small ones."""
    big = (*lpgen.paper_lp(600, 800, seed=1), capi.LP_MAX_LE)  # 657 pivots
    lps = [big] + _small(24, seed=2)
    opt = capi.lp_options_default(solo_elems=200000, spill_pivots=40, lanes=lanes)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=256 << 20, max_slots=32)
    try:
        res, done = _run(srv, lps)
        spills, restores, host = capi.lp_server_spill_stats(srv)
        _, _, used, queued = capi.lp_server_stats(srv)
    finally:
        capi.lp_server_destroy(srv)
    assert spills >= 1 and restores == spills and host > 0
    assert used == 0 and queued == 0
    assert sum(d < done[0] for d in done[1:]) >= 12
    for lp, r in zip(lps, res):
        _same_as_oracle(lp, r)


def test_fp64_spilled_lp_stops_at_the_iteration_limit():
    """max_iters 130 with slices of 50: the slices are 50, 50 and 30 pivots
    and the LP ends in LP_ITER_LIMIT with the oracle's values after 130
    pivots."""
    big = (*lpgen.paper_lp(500, 700, seed=3), capi.LP_MAX_LE)  # 853 pivots
    lps = [big] + _small(12, seed=4)
    opt = capi.lp_options_default(solo_elems=200000, spill_pivots=50, max_iters=130)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=256 << 20, max_slots=16)
    try:
        res, _ = _run(srv, lps)
    finally:
        capi.lp_server_destroy(srv)
    assert res[0][1] == capi.LP_ITER_LIMIT and res[0][2] == 130
    _same_as_oracle(big, res[0], max_iters=130)
    for lp, r in zip(lps[1:], res[1:]):
        _same_as_oracle(lp, r)


def test_fp64_two_large_lps_take_turns():
    """Two large LPs and small ones interleaved: while one is spilled the
    other runs (two handles hold their host-side states); primal and dual
    form; the oracle's bits."""
    A1, b1, c1 = lpgen.paper_lp(450, 600, seed=5)  # 371 pivots
    A2, b2, c2 = lpgen.dual_of(*lpgen.paper_lp(500, 400, seed=6))  # 102 pivots
    sm = _small(16, seed=7)
    lps = [(A1, b1, c1, capi.LP_MAX_LE)] + sm[:8] + [(A2, b2, c2, capi.LP_MIN_GE)] + sm[8:]
    opt = capi.lp_options_default(solo_elems=200000, spill_pivots=25)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=256 << 20, max_slots=16)
    try:
        res, _ = _run(srv, lps)
        spills, restores, _ = capi.lp_server_spill_stats(srv)
    finally:
        capi.lp_server_destroy(srv)
    assert spills >= 2 and restores == spills
    for lp, r in zip(lps, res):
        _same_as_oracle(lp, r)


def _serve32(lps, budget, slots, spill, solo=-1, k=20):
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=k, spill_pivots=spill,
                                  solo_elems=solo)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=budget, max_slots=slots)
    try:
        res, _ = _run(srv, lps)
        return res, capi.lp_server_spill_stats(srv), capi.lp_server_stats(srv)
    finally:
        capi.lp_server_destroy(srv)


def _same32(a, b):
    assert a[1] == b[1] and a[2] == b[2]
    assert _bits([a[0]])[0] == _bits([b[0]])[0]
    assert np.array_equal(_bits(a[3]), _bits(b[3])) and np.array_equal(_bits(a[4]), _bits(b[4]))


def test_fp32_rounds_spill_under_a_small_budget():
    """Twelve LPs of 250-400 rows under a budget that holds two: LPs are
    spilled between rounds and readmitted; each result has the bits it has
    on a server with room for all twelve, and reaches the oracle's optimum
    within 1e-6."""
    lps = [(*lpgen.paper_lp(m, n, seed=40 + k), capi.LP_MAX_LE)
           for k, (m, n) in enumerate(lpgen.log_uniform_shapes(12, 250, 400, 8))]
    ref, sp0, _ = _serve32(lps, 1 << 30, 32, 0)
    assert sp0[0] == 0
    res, (spills, restores, host), (done, _, used, queued) = _serve32(lps, 6 << 20, 8, 20)
    assert spills >= 4 and restores == spills and host > 0
    assert done == len(lps) and used == 0 and queued == 0
    for lp, a, b in zip(lps, res, ref):
        _same32(a, b)
        o = oracle.solve(lp[0], lp[1], lp[2], sense=lp[3])
        assert a[1] == capi.LP_OPTIMAL
        assert abs(a[0] - o.obj) / max(1.0, abs(o.obj)) <= 1e-6


def test_fp32_rounds_make_way_for_a_large_lp():
    """FP32 rounds with a large LP (which runs alone) behind them: once every
    LP in the rounds has made spill_pivots pivots they are spilled, the large
    LP runs, and they come back; every result has the bits of the server
    that does not spill."""
    lps = [(*lpgen.paper_lp(m, n, seed=60 + k), capi.LP_MAX_LE)
           for k, (m, n) in enumerate(lpgen.log_uniform_shapes(6, 200, 300, 9))]
    lps.insert(3, (*lpgen.paper_lp(500, 700, seed=3), capi.LP_MAX_LE))
    ref, _, _ = _serve32(lps, 1 << 30, 16, 0, solo=200000)
    res, (spills, restores, _), _ = _serve32(lps, 1 << 30, 16, 20, solo=200000)
    assert spills >= 1 and restores == spills
    for a, b in zip(res, ref):
        _same32(a, b)
