"""Batched solves: many uneven LPs in one persistent launch.

Every LP of a batch must give, bit for bit, what the FP64 oracle gives for it
alone (status, pivot count, objective, x, y): the batch runs the single-LP
pivot code on groups of CTAs, so mixing LPs changes nothing per LP.
"""
import os

import numpy as np
import pytest

import oracle
from golden_io import read_lp
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


def _mixed(count, lo, hi, seed):
    lps = []
    for k, (m, n) in enumerate(lpgen.log_uniform_shapes(count, lo, hi, seed)):
        A, b, c = lpgen.dense_lp(m, n, seed=1000 * seed + k)
        if k % 3 == 2:
            lps.append((*lpgen.dual_of(A, b, c), capi.LP_MIN_GE))
        else:
            lps.append((A, b, c, capi.LP_MAX_LE))
    return lps


def _check_against_oracle(lps, res):
    obj, st, it, xs, ys = res
    for k, (A, b, c, sense) in enumerate(lps):
        o = oracle.solve(A, b, c, sense=sense)
        assert st[k] == o.status and it[k] == o.iters, k
        assert _bits([obj[k]])[0] == _bits([o.obj])[0], (k, obj[k], o.obj)
        assert np.array_equal(_bits(xs[k]), _bits(o.x)), k
        assert np.array_equal(_bits(ys[k]), _bits(o.y)), k


@pytest.mark.parametrize("group_elems,threads", [(0, 0), (4096, 128), (20000, 512), (1 << 30, 256)])
def test_batch_bitwise_vs_oracle(group_elems, threads):
    lps = _mixed(48, 4, 160, seed=1)
    opt = capi.lp_options_default(group_elems=group_elems, threads=threads)
    _check_against_oracle(lps, capi.lp_solve_batch(lps, opt, want_xy=True))
    if group_elems == 4096:
        assert capi.lp_batch_stats()[4] > 1  # some LP ran on a multi-CTA group


def test_batch_config_shapes_vs_oracle():
    """m, n log-uniform in [32, 1024] like the batched workload."""
    lps = _mixed(96, 32, 1024, seed=2)
    _check_against_oracle(lps, capi.lp_solve_batch(lps, want_xy=True))


def test_batch_golden_and_degenerate_members():
    lps = []
    for name in ("chvatal_cycling.txt", "beale_cycling.txt", "wyndor.txt", "bland_tie.txt"):
        g = read_lp(name)
        lps.append((g["A"], g["b"], g["c"], capi.LP_MAX_LE))
    lps.append((np.array([[1.0, -1.0], [2.0, 0.0]]), np.array([4.0, 6.0]), np.array([1.0, 3.0]),
                capi.LP_MAX_LE))  # unbounded
    lps.append((np.array([[-1.0, -2.0]]), np.array([1.0]), np.array([1.0, 1.0]),
                capi.LP_MIN_GE))  # infeasible
    lps += _mixed(10, 3, 40, seed=3)
    _check_against_oracle(lps, capi.lp_solve_batch(lps, want_xy=True))


def test_batch_device_inputs_and_repeat():
    torch = pytest.importorskip("torch")
    lps = _mixed(20, 16, 300, seed=4)
    dev = [(torch.from_numpy(A).cuda(), torch.from_numpy(b).cuda(), torch.from_numpy(c).cuda(), s)
           for A, b, c, s in lps]
    r1 = capi.lp_solve_batch(dev, want_xy=True)
    r2 = capi.lp_solve_batch(lps, want_xy=True)
    for a, b2 in zip(r1[:3], r2[:3]):
        assert np.array_equal(np.asarray(a), np.asarray(b2))
    _check_against_oracle(lps, r1)


def test_batch_errors_name_the_lp():
    lps = _mixed(5, 4, 20, seed=5)
    A, b, c, _ = lps[3]
    bad = b.copy()
    bad[0] = -1.0
    lps[3] = (A, bad, c, capi.LP_MAX_LE)
    with pytest.raises(capi.LpError) as e:
        capi.lp_solve_batch(lps)
    assert e.value.code == capi.LP_ERR_INFEASIBLE_START and "LP 3" in str(e.value)


def test_batch_autotune_and_cache(tmp_path):
    lps = _mixed(32, 16, 400, seed=6)
    cache = str(tmp_path / "tune.txt")
    best = capi.lp_batch_autotune(lps, cache_path=cache)
    assert best.group_elems in (16384, 65536, 262144, 1048576) and best.threads in (256, 512)
    again = capi.lp_batch_autotune(lps, cache_path=cache)  # cache hit
    assert (again.group_elems, again.threads) == (best.group_elems, best.threads)
    assert len(open(cache).read().strip().splitlines()) == 1
    _check_against_oracle(lps, capi.lp_solve_batch(lps, best, want_xy=True))


def _rel(a, b):
    return abs(a - b) / max(1.0, abs(b))


@pytest.mark.parametrize("k", [50, 200])
def test_batch_fp32_objective_vs_fp64_oracle(k):
    """FP32 tableaus with FP64 reinversion every k pivots, many LPs in one
    batch: each objective within 1e-6 of the FP64 oracle, with an FP64
    optimality certificate for the x, y returned."""
    lps = _mixed(40, 16, 400, seed=7)
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=k)
    obj, st, it, xs, ys = capi.lp_solve_batch(lps, opt, want_xy=True)
    for j, (A, b, c, sense) in enumerate(lps):
        o = oracle.solve(A, b, c, sense=sense)
        assert st[j] == capi.LP_OPTIMAL, j
        assert _rel(obj[j], o.obj) <= 1e-6, (j, obj[j], o.obj)
        cert = oracle.certificate(A, b, c, xs[j], ys[j], obj[j], sense=sense)
        scale = max(1.0, abs(o.obj), float(np.max(np.abs(b))), float(np.max(np.abs(c))))
        assert max(cert.values()) <= 1e-6 * scale, (j, cert)


def test_batch_fp32_matches_solo_fp32():
    """A batched FP32 LP pivots, reinverts and ends exactly as it does alone."""
    lps = _mixed(12, 8, 200, seed=8)
    opt = capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50)
    obj, st, it = capi.lp_solve_batch(lps, opt)
    for j, (A, b, c, sense) in enumerate(lps):
        h = capi.lp_create(capi.lp_options_default(precision=capi.LP_FP32_REINV, reinv_k=50))
        try:
            capi.lp_load(h, A, b, c, sense)
            capi.lp_solve(h)
            o1, s1, i1 = capi.lp_result(h)
        finally:
            capi.lp_destroy(h)
        assert (st[j], it[j]) == (s1, i1), j
        assert _bits([obj[j]])[0] == _bits([o1])[0], (j, obj[j], o1)
