"""The allocation-free entry point, lp_solve_noalloc, against the regular
handle-based path (lp_create / lp_load / lp_solve / lp_result).

lp_solve_noalloc serves callers that cannot allocate device memory when they
solve (a fixed memory budget handed out up front, a host process that owns
the allocator, loops that must not pay an allocation's latency): it keeps all
of its working memory in one fixed device array.  Both paths run the same
FP64 kernels, so the results must agree bit for bit -- the tolerance the other
FP64 parity tests use.  Two different LPs in a row check that the shared array
carries nothing over from one call to the next.  A wide min-form LP puts the
per-CTA selection scratch into the array too (it does not fit shared
memory), and device free memory is unchanged across repeated calls.  This
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_1804_04737_gb300 import capi, lpgen
from paper_1804_04737_gb300.build import build_library

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    build_library()
    capi.load_library()


def _bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


def _regular(A, b, c, sense):
    m, n = A.shape
    h = capi.lp_create()
    try:
        capi.lp_load(h, A, b, c, sense)
        capi.lp_solve(h)
        x, y = np.empty(n), np.empty(m)
        obj, st, it = capi.lp_result(h, x, y)
        return obj, st, it, x, y
    finally:
        capi.lp_destroy(h)


def _noalloc(A, b, c, sense):
    m, n = A.shape
    x, y = np.full(n, np.nan), np.full(m, np.nan)
    obj, st, it = capi.lp_solve_noalloc(A, b, c, sense, x=x, y=y)
    return obj, st, it, x, y


def test_noalloc_matches_regular_two_calls_in_a_row():
    cases = [(lpgen.dense_lp(700, 900, seed=21), capi.LP_MAX_LE),
             (lpgen.dual_of(*lpgen.dense_lp(300, 250, seed=22)), capi.LP_MIN_GE),
             (lpgen.dense_lp(64, 64, seed=0), capi.LP_MAX_LE)]
    for (A, b, c), sense in cases:
        ref = _regular(A, b, c, sense)
        got = _noalloc(A, b, c, sense)
        assert got[1] == ref[1] == capi.LP_OPTIMAL
        assert got[2] == ref[2]
        assert _bits([got[0]])[0] == _bits([ref[0]])[0]
        assert np.array_equal(_bits(got[3]), _bits(ref[3]))
        assert np.array_equal(_bits(got[4]), _bits(ref[4]))


def test_noalloc_device_buffers_and_size_limit():
    torch = pytest.importorskip("torch")
    A, b, c = lpgen.dense_lp(500, 400, seed=23)
    ref = _regular(A, b, c, capi.LP_MAX_LE)
    tA, tb, tc = (torch.from_numpy(v).cuda() for v in (A, b, c))
    x = torch.empty(400, dtype=torch.float64, device="cuda")
    y = torch.empty(500, dtype=torch.float64, device="cuda")
    obj, st, it = capi.lp_solve_noalloc(tA, tb, tc, capi.LP_MAX_LE, x=x, y=y)
    assert (st, it) == (ref[1], ref[2]) and obj == ref[0]
    assert np.array_equal(_bits(x.cpu().numpy()), _bits(ref[3]))
    assert np.array_equal(_bits(y.cpu().numpy()), _bits(ref[4]))
    big = np.ones((2048, 2048))
    with pytest.raises(capi.LpError) as e:
        capi.lp_solve_noalloc(big, np.ones(2048), np.ones(2048))
    assert e.value.code == capi.LP_ERR_INVALID_ARG and "64 MiB" in str(e.value)


def test_noalloc_scratch_in_the_array_bitwise():
    """A min-form LP with 26101 tableau columns: its per-CTA selection scratch
    (a row of keys, 209 KB) exceeds shared memory, so the solve keeps it in
    the array as well (about 59 MB of the 64 MiB in all)."""
    A, b, c = lpgen.dual_of(*lpgen.dense_lp(26000, 100, seed=24))
    assert A.shape == (100, 26000)
    ref = _regular(A, b, c, capi.LP_MIN_GE)
    for _ in range(2):
        got = _noalloc(A, b, c, capi.LP_MIN_GE)
        assert got[1] == ref[1] == capi.LP_OPTIMAL and got[2] == ref[2]
        assert _bits([got[0]])[0] == _bits([ref[0]])[0]
        assert np.array_equal(_bits(got[3]), _bits(ref[3]))
        assert np.array_equal(_bits(got[4]), _bits(ref[4]))


def test_noalloc_leaves_device_memory_unchanged():
    """Repeated calls take no device memory: the free memory the driver reports
    is the same before and after (after one call that loads the array)."""
    torch = pytest.importorskip("torch")
    A, b, c = lpgen.dense_lp(600, 800, seed=25)
    first = _noalloc(A, b, c, capi.LP_MAX_LE)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(4):
        got = _noalloc(A, b, c, capi.LP_MAX_LE)
        assert got[:3] == first[:3]
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
