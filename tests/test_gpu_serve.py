"""Serving with continuous batching, through the C ABI.

Requests are submitted while others are on the GPU; every result must equal
the FP64 oracle's for that LP alone, bit for bit (each LP runs the single-LP
pivot code on its own group of CTAs), whatever else is in the mix, under a
budget that forces requests to wait for memory, and across kernel relaunches.
"""
import os
import threading
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


def _mix(count, lo, hi, seed):
    out = []
    for k, (m, n) in enumerate(lpgen.log_uniform_shapes(count, lo, hi, seed)):
        A, b, c = lpgen.dense_lp(m, n, seed=7000 * seed + k)
        out.append((*lpgen.dual_of(A, b, c), capi.LP_MIN_GE) if k % 4 == 3
                   else (A, b, c, capi.LP_MAX_LE))
    return out


def _check(lp, res):
    A, b, c, sense = lp
    obj, st, it, x, y, lat = res
    o = oracle.solve(A, b, c, sense=sense)
    assert st == o.status and it == o.iters
    assert _bits([obj])[0] == _bits([o.obj])[0]
    assert np.array_equal(_bits(x), _bits(o.x)) and np.array_equal(_bits(y), _bits(o.y))
    assert lat > 0.0


LANES = pytest.mark.parametrize("lanes", [0, 3])  # the server kernel, or three lanes


@LANES
def test_serve_stream_matches_oracle(lanes):
    lps = _mix(60, 8, 600, seed=1)
    srv = capi.lp_server_create(capi.lp_options_default(lanes=lanes), hbm_budget_bytes=2 << 30,
                                max_slots=64)
    try:
        tickets = []
        for k, lp in enumerate(lps):  # staggered arrivals: new requests join running ones
            tickets.append(capi.lp_server_submit(srv, *lp))
            if k % 7 == 0:
                time.sleep(0.002)
        for lp, t in zip(lps, tickets):
            _check(lp, capi.lp_server_wait(srv, t, lp[0].shape[0], lp[0].shape[1]))
        assert capi.lp_server_stats(srv)[0] == len(lps)
    finally:
        capi.lp_server_destroy(srv)


@LANES
def test_serve_small_budget_admission_and_threads(lanes):
    """A budget that holds only a few tableaus: requests wait for memory (with
    lanes, LPs a 4 MB slice cannot hold run alone on the whole 12 MB)."""
    lps = _mix(24, 100, 400, seed=2)
    srv = capi.lp_server_create(capi.lp_options_default(lanes=lanes), hbm_budget_bytes=12 << 20,
                                max_slots=8)
    results = {}
    try:
        def client(idx):
            for k in idx:
                t = capi.lp_server_submit(srv, *lps[k])
                results[k] = capi.lp_server_wait(srv, t, lps[k][0].shape[0], lps[k][0].shape[1])
        ths = [threading.Thread(target=client, args=(range(j, len(lps), 4),)) for j in range(4)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
        for k, lp in enumerate(lps):
            _check(lp, results[k])
        _, _, used, queued = capi.lp_server_stats(srv)
        assert used == 0 and queued == 0
    finally:
        capi.lp_server_destroy(srv)


@LANES
def test_serve_idle_relaunch_and_rejected_request(lanes):
    srv = capi.lp_server_create(capi.lp_options_default(lanes=lanes), hbm_budget_bytes=1 << 30,
                                max_slots=16)
    try:
        lp = _mix(1, 50, 60, seed=3)[0]
        _check(lp, capi.lp_server_wait(srv, capi.lp_server_submit(srv, *lp), lp[0].shape[0], lp[0].shape[1]))
        time.sleep(0.3)  # the kernel ends after its idle period
        A, b, c, _ = _mix(1, 20, 30, seed=4)[0]
        bad = b.copy()
        bad[2] = -5.0
        tb = capi.lp_server_submit(srv, A, bad, c)
        lp2 = _mix(1, 70, 80, seed=5)[0]
        t2 = capi.lp_server_submit(srv, *lp2)
        with pytest.raises(capi.LpError) as e:
            capi.lp_server_wait(srv, tb, A.shape[0], A.shape[1])
        assert e.value.code == capi.LP_ERR_INFEASIBLE_START
        _check(lp2, capi.lp_server_wait(srv, t2, lp2[0].shape[0], lp2[0].shape[1]))
        assert capi.lp_server_stats(srv)[1] >= 2  # relaunched after the idle exit
    finally:
        capi.lp_server_destroy(srv)


@LANES
def test_serve_large_lps_alone_in_the_mix(lanes):
    """LPs of at least solo_elems tableau elements run alone on the single-LP
    kernels, between busy periods of the persistent kernel; with a low
    threshold about half of a mixed stream does.  Every result is still the
    oracle's, bit for bit, and rejected large requests get the kernel's
    verdicts."""
    lps = _mix(40, 8, 300, seed=6)
    opt = capi.lp_options_default(solo_elems=20000, lanes=lanes)
    solo = sum((lp[0].shape[0] + 1) * (-(-(sum(lp[0].shape) + 1) // 32) * 32) >= 20000
               for lp in lps)
    assert 5 <= solo <= 35
    srv = capi.lp_server_create(opt, hbm_budget_bytes=1 << 30, max_slots=32)
    try:
        A, b, c, _ = _mix(1, 150, 160, seed=8)[0]
        bad = b.copy()
        bad[3] = -1.0
        nan = c.copy()
        nan[0] = np.nan
        tickets = []
        for k, lp in enumerate(lps):
            tickets.append(capi.lp_server_submit(srv, *lp))
            if k == 10:
                tb = capi.lp_server_submit(srv, A, bad, c)
                tn = capi.lp_server_submit(srv, A, b, nan)
            if k % 5 == 0:
                time.sleep(0.002)
        for lp, t in zip(lps, tickets):
            _check(lp, capi.lp_server_wait(srv, t, lp[0].shape[0], lp[0].shape[1]))
        for t, code in ((tb, capi.LP_ERR_INFEASIBLE_START), (tn, capi.LP_ERR_INVALID_ARG)):
            with pytest.raises(capi.LpError) as e:
                capi.lp_server_wait(srv, t, A.shape[0], A.shape[1])
            assert e.value.code == code
        done, launches, used, queued = capi.lp_server_stats(srv)
        assert done == len(lps) + 2 and used == 0 and queued == 0
        assert launches >= solo + 1
    finally:
        capi.lp_server_destroy(srv)


# ---- FP32 tableaus with FP64 reinversion ----

OBJ_TOL32 = 1e-6


def _serve32(lps, budget=2 << 30, slots=64, k=50, stagger=True):
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=k)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=budget, max_slots=slots)
    try:
        tickets = []
        for i, lp in enumerate(lps):
            tickets.append(capi.lp_server_submit(srv, *lp))
            if stagger and i % 7 == 0:
                time.sleep(0.002)
        res = [capi.lp_server_wait(srv, t, lp[0].shape[0], lp[0].shape[1])
               for lp, t in zip(lps, tickets)]
        return res, capi.lp_server_stats(srv)
    finally:
        capi.lp_server_destroy(srv)


def test_serve_fp32_objective_and_mix_invariance():
    """FP32 serving: requests join running rounds; every result reaches the
    FP64 optimum within the FP32 mode's tolerance with an FP64 certificate,
    and each result is the same, bit for bit, served alone or in the mix."""
    lps = _mix(40, 8, 600, seed=3)
    res, stats = _serve32(lps)
    assert stats[0] == len(lps) and stats[1] >= 1
    for lp, r in zip(lps, res):
        A, b, c, sense = lp
        obj, st, it, x, y, lat = r
        o = oracle.solve(A, b, c, sense=sense)
        assert st == capi.LP_OPTIMAL and lat > 0.0
        assert abs(obj - o.obj) / max(1.0, abs(o.obj)) <= OBJ_TOL32, (obj, o.obj)
        cert = oracle.certificate(A, b, c, x, y, obj, sense=sense)
        scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
        assert max(cert.values()) <= 1e-9 * scale * 1e3, cert
    for i in (0, 7, 19, 33):
        (alone,), _ = _serve32([lps[i]], stagger=False)
        assert _bits([alone[0]])[0] == _bits([res[i][0]])[0]
        assert alone[1] == res[i][1] and alone[2] == res[i][2]
        assert np.array_equal(_bits(alone[3]), _bits(res[i][3]))
        assert np.array_equal(_bits(alone[4]), _bits(res[i][4]))


def test_serve_fp32_large_lps_alone():
    """FP32 serving with a low solo_elems: the large LPs leave the rounds and
    run alone as lp_load + lp_solve run them, bit for bit, between rounds;
    every result still reaches the FP64 optimum within the FP32 tolerance."""
    lps = _mix(24, 8, 300, seed=6)
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50, solo_elems=20000)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=1 << 30, max_slots=32)
    try:
        tickets = [capi.lp_server_submit(srv, *lp) for lp in lps]
        res = [capi.lp_server_wait(srv, t, lp[0].shape[0], lp[0].shape[1])
               for lp, t in zip(lps, tickets)]
        assert capi.lp_server_stats(srv)[2] == 0
    finally:
        capi.lp_server_destroy(srv)
    alone = 0
    h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50))
    try:
        for lp, r in zip(lps, res):
            A, b, c, sense = lp
            o = oracle.solve(A, b, c, sense=sense)
            assert r[1] == capi.LP_OPTIMAL
            assert abs(r[0] - o.obj) / max(1.0, abs(o.obj)) <= OBJ_TOL32, (r[0], o.obj)
            m, n = A.shape
            if (m + 1) * (-(-(m + n + 1) // 32) * 32) < 20000:
                continue
            alone += 1
            capi.lp_load(h, A, b, c, sense)
            capi.lp_solve(h)
            x, y = np.empty(n), np.empty(m)
            obj, st, it = capi.lp_result(h, x, y)
            assert _bits([obj])[0] == _bits([r[0]])[0] and st == r[1] and it == r[2]
            assert np.array_equal(_bits(x), _bits(r[3])) and np.array_equal(_bits(y), _bits(r[4]))
    finally:
        capi.lp_destroy(h)
    assert alone >= 3


def test_serve_fp32_small_budget_and_rejects():
    """A budget that holds a few LPs at a time (requests wait for memory
    between rounds), reinv_k = 200, and a request the FP32 mode refuses."""
    lps = _mix(12, 100, 400, seed=4)
    res, stats = _serve32(lps, budget=24 << 20, slots=8, k=200)
    assert stats[0] == len(lps)
    for lp, r in zip(lps, res):
        o = oracle.solve(lp[0], lp[1], lp[2], sense=lp[3])
        assert r[1] == capi.LP_OPTIMAL
        assert abs(r[0] - o.obj) / max(1.0, abs(o.obj)) <= OBJ_TOL32
    A, b, c = lpgen.dense_lp(30, 40, seed=9)
    bad = b.copy()
    bad[3] = -1.0
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV)
    srv = capi.lp_server_create(opt, hbm_budget_bytes=64 << 20, max_slots=4)
    try:
        t = capi.lp_server_submit(srv, A, bad, c)
        t2 = capi.lp_server_submit(srv, A, b, c)
        with pytest.raises(capi.LpError) as e:
            capi.lp_server_wait(srv, t, 30, 40)
        assert e.value.code == capi.LP_ERR_INFEASIBLE_START
        r = capi.lp_server_wait(srv, t2, 30, 40)
        assert r[1] == capi.LP_OPTIMAL
    finally:
        capi.lp_server_destroy(srv)
