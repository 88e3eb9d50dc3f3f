"""The C-ABI library loads and exports every entry point its header declares
(no GPU needed: only symbol lookup and pure host calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1804_04737_gb300 import capi
from paper_1804_04737_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    hdr_dir = os.path.join(ROOT, "include")
    for f in os.listdir(hdr_dir):
        if f.endswith(".h"):
            src = open(os.path.join(hdr_dir, f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(lp_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    build_library()
    return capi.load_library()


def test_every_declared_symbol_exported(lib):
    names = _declared()
    assert {"lp_create", "lp_load", "lp_solve", "lp_result", "lp_destroy"} <= names
    raw = ctypes.CDLL(capi.LIB_PATH)
    for name in sorted(names):
        assert hasattr(raw, name), name


def test_binding_covers_header(lib):
    bound = {s[0] for s in capi._SIGS}
    assert _declared() <= bound, _declared() - bound


def test_options_layout_and_defaults(lib):
    assert lib.lp_options_size() == ctypes.sizeof(capi.lp_options)
    o = capi.lp_options_default()
    assert o.precision == capi.LP_FP64 and o.bland_after == 32 and o.reinv_k == 50
    assert o.max_iters >= 10 ** 12 and o.spin_timeout_cycles > 0 and o.trace_cap == 0
    assert capi.lp_version().startswith("gbsimplex")


def test_null_arguments_rejected_without_gpu(lib):
    assert lib.lp_create(None, None) == capi.LP_ERR_INVALID_ARG
    assert lib.lp_load(None, 1, 1, None, None, None, 0) == capi.LP_ERR_INVALID_ARG
    assert lib.lp_solve(None) == capi.LP_ERR_INVALID_ARG
    lib.lp_destroy(None)
    assert "NULL" in capi.lp_last_error(None)


def test_server_options_checked_without_gpu(lib):
    """The server's option checks come before any CUDA call: lanes outside
    0..16 and a negative spill_pivots are refused; the stats calls refuse
    NULL; no product has run, so no MMA is counted."""
    import ctypes
    srv = ctypes.c_void_p()
    for bad in ({"lanes": 17}, {"lanes": -1}, {"spill_pivots": -1}):
        opt = capi.lp_options_default(**bad)
        assert lib.lp_server_create(ctypes.byref(srv), ctypes.byref(opt), 1 << 30, 8) == \
            capi.LP_ERR_INVALID_ARG
        assert not srv.value
    assert lib.lp_server_spill_stats(None, None, None, None) == capi.LP_ERR_INVALID_ARG
    assert lib.lp_dgemm_stats(None) == capi.LP_ERR_INVALID_ARG
    assert capi.lp_dgemm_stats() == 0
    o = capi.lp_options_default()
    assert o.lanes == 3 and o.spill_pivots == 0 and o.zero_skip == 1


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        capi.load_library(str(tmp_path / "nope.so"))


def test_noalloc_binding_checks_shapes():
    """The binding rejects inconsistent shapes before calling the library (a
    short b or c would be read past its end, a short x or y written past it)."""
    A = np.ones((3, 4))
    for kw in ({"b": np.ones(2)}, {"c": np.ones(5)}, {"x": np.ones(3)}, {"y": np.ones(4)}):
        args = {"b": np.ones(3), "c": np.ones(4), **kw}
        x, y = args.pop("x", None), args.pop("y", None)
        with pytest.raises(ValueError):
            capi.lp_solve_noalloc(A, args["b"], args["c"], x=x, y=y)
