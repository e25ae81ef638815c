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


def test_unbuilt_context_host_checks(lib):
    """A created but unbuilt context: queries that need no model answer, everything that
    needs the built model returns NOT_BUILT, and argument checks come before any CUDA call."""
    import numpy as np

    import paper_2502_05635_gb300 as tg
    import workloads as wl
    D = ct.POINTER(ct.c_double)
    buf = (ct.c_double * 64)()
    dp = ct.cast(buf, D)
    h = ct.c_void_p()
    d = tg.model_desc(wl.small_model(4, 1))
    assert lib.tdagw_create(ct.byref(d), None, ct.byref(h)) == tg.OK
    try:
        N, Nb, Nk = ct.c_int64(), ct.c_int(), ct.c_int()
        assert lib.tdagw_model_info(h, ct.byref(N), ct.byref(Nb), ct.byref(Nk)) == tg.OK
        assert (N.value, Nb.value, Nk.value) == (64, 2, 16)
        rows = (ct.c_int64 * 1)(0)
        assert lib.tdagw_get_model(h, None, None, None, None, None) == tg.ERR_NOT_BUILT
        assert "tdagw_build_kernel" in tg.tdagw_last_error()
        assert lib.tdagw_get_kernel_entries(h, rows, rows, 1, dp) == tg.ERR_NOT_BUILT
        assert lib.tdagw_compress_svd(h, 4, 0, 0, 1, 0) == tg.ERR_NOT_BUILT
        assert lib.tdagw_set_factors(h, 1, dp, dp, dp, None) == tg.ERR_NOT_BUILT
        assert lib.tdagw_compress_channels(h, 1, 0, 0, 1, 0.0) == tg.ERR_NOT_BUILT
        # dense diagonal channels given: the layout still needs the built model's sizes
        assert lib.tdagw_set_channel_factors(h, 0, None, None, None, None, dp) == tg.ERR_NOT_BUILT
        x = (ct.c_double * 8)()
        y = (ct.c_double * 8)()
        assert lib.tdagw_apply(h, tg.FULL, ct.cast(x, ct.c_void_p), ct.cast(y, ct.c_void_p)) == tg.ERR_NOT_BUILT
        f = tg.Field(kind=1, E0=1e-3, dir_x=1.0)
        st = (ct.c_int * 1)(4)
        assert lib.tdagw_propagate(h, ct.byref(f), 1, st, 0.2, tg.FULL, 0) == tg.ERR_NOT_BUILT
        assert lib.tdagw_adjoint(h, dp, None, None) == tg.ERR_NOT_BUILT
        step = ct.c_int64(-1)
        assert lib.tdagw_get_state(h, None, None, ct.byref(step)) == tg.ERR_NOT_BUILT
        assert lib.tdagw_set_state(h, dp, None, 0) == tg.ERR_NOT_BUILT
        # factor queries: no factors yet
        r = ct.c_int(-1)
        assert lib.tdagw_get_factors(h, ct.byref(r), None, None, None, None) == tg.OK and r.value == 0
        assert lib.tdagw_get_factors(h, ct.byref(r), dp, None, None, None) == tg.ERR_NO_FACTORS
        r.value = -1
        assert lib.tdagw_get_channel_factors(h, ct.byref(r), None, None, None, None, None) == tg.OK
        assert r.value == 0
        assert lib.tdagw_get_channel_factors(h, ct.byref(r), None, dp, None, None, None) == tg.ERR_NO_FACTORS
        nrows = ct.c_int64(-1)
        assert lib.tdagw_observables(h, None, 0, ct.byref(nrows), 1) == tg.OK and nrows.value == 0
        # the K^diag switch is a host flag
        assert lib.tdagw_set_kdiag_blocks(h, 2) == tg.ERR_INVALID_ARG
        assert lib.tdagw_set_kdiag_blocks(h, 1) == tg.OK
        assert lib.tdagw_set_kdiag_blocks(h, 0) == tg.OK
        # propagate argument checks come after the build check
        assert lib.tdagw_propagate(h, ct.byref(f), 0, st, 0.2, tg.FULL, 0) == tg.ERR_NOT_BUILT
    finally:
        lib.tdagw_destroy(h)


def test_hhg_and_noalloc_argument_checks(lib):
    """Host-side checks of the two context-free entry points (no pointer is dereferenced)."""
    import paper_2502_05635_gb300 as tg
    D = ct.POINTER(ct.c_double)
    J = ct.cast((ct.c_double * 16)(), D)
    w = ct.cast((ct.c_double * 2)(), D)
    out = ct.cast((ct.c_double * 2)(), D)
    st = (ct.c_int * 1)(5)
    # rows must cover steps + 1 recorded samples
    assert lib.tdagw_hhg_spectrum(J, 3, 1, 1, st, 0.2, w, 2, out, None) == tg.ERR_INVALID_ARG
    assert "rows" in tg.tdagw_last_error()
    neg = (ct.c_int * 1)(-1)
    assert lib.tdagw_hhg_spectrum(J, 6, 1, 1, neg, 0.2, w, 2, out, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_hhg_spectrum(J, 6, 1, 1, st, 0.0, w, 2, out, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_hhg_spectrum(J, 6, 0, 1, st, 0.2, w, 2, out, None) == tg.ERR_INVALID_ARG
    assert lib.tdagw_hhg_spectrum(J, 6, 1, 65536, st, 0.2, w, 2, out, None) == tg.ERR_INVALID_ARG
    assert "65535" in tg.tdagw_last_error()
    # allocation-free apply: addresses are only checked, never read
    a16, b16, s16, odd = 0x10000, 0x20000, 0x30000, 0x10008
    f = lib.tdagw_apply_lowrank_noalloc
    assert f(None, b16, 8, s16, s16, 64, 8, a16, b16, None) == tg.ERR_INVALID_ARG
    assert f(a16, b16, 8, s16, s16, 0, 8, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert f(a16, b16, 8, s16, s16, 64, 0, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert f(a16, b16, 8, s16, s16, 64, 4096, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert f(a16, b16, 7, s16, s16, 64, 6, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert f(a16, b16, 4, s16, s16, 64, 6, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert f(odd, b16, 8, s16, s16, 64, 8, a16 + 0x100, b16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert "aligned" in tg.tdagw_last_error()
    assert f(a16, b16, 8, s16, s16, 64, 8, a16 + 0x100, a16 + 0x100, None) == tg.ERR_INVALID_ARG
    assert "alias" in tg.tdagw_last_error()


def test_binding_checks_shapes_before_passing_pointers(lib):
    """The binding checks array shapes, dtypes and counts (the C side cannot see extents);
    a created but unbuilt context answers model_info, so no GPU is needed."""
    import numpy as np
    import torch

    import paper_2502_05635_gb300 as tg
    import workloads as wl

    h = tg.tdagw_create(tg.model_desc(wl.small_model(4, 1)))   # N = 64, Nb = 2, Nk = 16, P = 4

    def bad(fn, *args, match="", **kw):
        with pytest.raises(tg.TdagwError) as e:
            fn(*args, **kw)
        assert e.value.code == tg.ERR_INVALID_ARG and match in str(e.value), str(e.value)

    try:
        c = np.zeros
        bad(tg.tdagw_set_factors, h, c((63, 4), complex), c(4), c((63, 4), complex), match="U must be")
        bad(tg.tdagw_set_factors, h, c((64, 4), complex), c(4), c((64, 5), complex), match="V must")
        bad(tg.tdagw_set_factors, h, c((64, 4), complex), c(3), c((64, 4), complex), match="S must")
        bad(tg.tdagw_set_factors, h, c((64, 4), complex), c(4), c((64, 4), complex), c(63, complex),
            match="64 entries")
        tg.tdagw_set_kdiag_blocks(h, 1)                            # blocks: Nk x P x P = 256
        bad(tg.tdagw_set_factors, h, c((64, 4), complex), c(4), c((64, 4), complex), c(64, complex),
            match="256 entries")
        tg.tdagw_set_kdiag_blocks(h, 0)
        U = c((4, 4, 16, 3), complex)
        bad(tg.tdagw_set_channel_factors, h, c((4, 4, 15, 3), complex), c((4, 4, 3)), U, match="U must be")
        bad(tg.tdagw_set_channel_factors, h, U, c((4, 4, 2)), U, match="S must")
        bad(tg.tdagw_set_channel_factors, h, U, c((4, 4, 3)), U, c((4, 16, 15), complex), match="D must")
        bad(tg.tdagw_set_channel_factors, h, U, c((4, 4, 3)), U, None, c((4, 3), int), match="ranks")
        bad(tg.tdagw_set_state, h, c(63, complex), match="N = 64")
        bad(tg.tdagw_set_state, h, c(64, complex), c(32, complex), match="N = 64")
        pulse = wl.Pulse()
        bad(tg.tdagw_propagate, h, [tg.make_field(pulse)] * 2, [10], 0.2, tg.FULL, match="step count")
        f = tg.make_field(pulse, table=c(20))
        bad(tg.tdagw_propagate, h, [f], [10], 0.2, tg.FULL, match="2 steps + 1")
        x = torch.zeros(64, dtype=torch.complex64)
        bad(tg.tdagw_apply, h, tg.FULL, torch.zeros(63, dtype=torch.complex64), x, match="64 elements")
        bad(tg.tdagw_apply, h, tg.FULL, torch.zeros(64, dtype=torch.complex128), x, match="complex64")
        bad(tg.tdagw_apply, h, tg.FULL, x, torch.zeros(64, dtype=torch.complex64), match="CUDA tensor")
        bad(tg.tdagw_adjoint, h, c((11, 1, 3)), 10, 1, match="last checkpointed")
        Ut = torch.zeros((64, 8), dtype=torch.complex64)
        S8 = torch.ones(8, dtype=torch.float32)
        nd = tg.tdagw_apply_lowrank_noalloc
        bad(nd, Ut, torch.zeros((64, 6), dtype=torch.complex64), S8, x, x.clone(), x.clone(), match="V must")
        bad(nd, Ut, Ut, torch.ones(9, dtype=torch.float32), x, x.clone(), x.clone(), match="rank <= ld")
        bad(nd, Ut, Ut, S8.double(), x, x.clone(), x.clone(), match="float32")
        bad(nd, Ut, Ut, S8, x, x.clone(), torch.zeros(65, dtype=torch.complex64), match="y must")
        bad(nd, Ut, Ut, S8, x, x.clone(), x.clone(), match="CUDA tensor")
        J = c((11, 2))
        bad(tg.tdagw_hhg_spectrum, J, [10], 0.2, np.ones(3), match="one step count")
        bad(tg.tdagw_hhg_spectrum, J, [10, 10], 0.2, np.ones(3), component=1, match="J must be")
        bad(tg.tdagw_hhg_spectrum, c((11, 2, 3)), [10, 10], 0.2, np.ones(3), component=3, match="component")
    finally:
        tg.tdagw_destroy(h)
