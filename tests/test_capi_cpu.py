"""The C-ABI library builds, loads and exports every symbol include/tdagw.h declares.

No GPU: only argument validation paths are exercised (they return error codes before any
CUDA call).
"""
import ctypes as ct
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tdagw.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tdagw_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2502_05635_gb300 as tg
    return tg.lib()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header(lib):
    import paper_2502_05635_gb300 as tg
    assert sorted(tg.EXPORTED) == _declared()
    for n in _declared():
        assert callable(getattr(tg, n)), n


def test_struct_layouts():
    import paper_2502_05635_gb300 as tg
    # int, int, double[4], 5 doubles, int (+ padding), double and int + 7 doubles + pointer
    assert ct.sizeof(tg.ModelDesc) == 4 + 4 + 32 + 40 + 8 + 8
    assert ct.sizeof(tg.Field) == 8 + 7 * 8 + 8


def test_invalid_arguments_return_codes(lib):
    import paper_2502_05635_gb300 as tg
    import workloads as wl
    h = ct.c_void_p()
    d = tg.model_desc(wl.small_model(0, 1))
    assert lib.tdagw_create(ct.byref(d), None, ct.byref(h)) == tg.ERR_INVALID_ARG
    assert "L must be" in tg.tdagw_last_error()
    d = tg.model_desc(wl.small_model(4, 3))
    assert lib.tdagw_create(ct.byref(d), None, ct.byref(h)) == tg.ERR_INVALID_ARG
    d = tg.model_desc(wl.small_model(4, 1), dtype=7)
    assert lib.tdagw_create(ct.byref(d), None, ct.byref(h)) == tg.ERR_INVALID_ARG
    assert lib.tdagw_create(None, None, ct.byref(h)) == tg.ERR_INVALID_ARG
    assert lib.tdagw_build_kernel(None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_apply(None, 0, None, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_propagate(None, None, 1, None, 0.2, 0, 0) == tg.ERR_INVALID_ARG
    assert lib.tdagw_compress_channels(None, 1, 0, 0, 1, 0.0) == tg.ERR_INVALID_ARG
    assert lib.tdagw_set_channel_factors(None, 0, None, None, None, None, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_get_channel_factors(None, None, None, None, None, None, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_hhg_spectrum(None, 1, 1, 1, None, 0.2, None, 1, None, None) == tg.ERR_INVALID_ARG
    lib.tdagw_destroy(None)


def test_package_fails_loudly_without_library(tmp_path, monkeypatch):
    import paper_2502_05635_gb300 as tg
    monkeypatch.setattr(tg, "_lib", None)
    monkeypatch.setattr(tg, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(tg.TdagwError):
        tg.lib()
