"""Allocation-free low-rank contraction (tdagw_apply_lowrank_noalloc) vs tdagw_apply.

For callers that cannot allocate device memory on their call path, the library offers a
variant of the low-rank apply that keeps its intermediate vectors in a fixed device array
instead of calling cudaMalloc.  These checks call it through the C ABI on caller-owned
arrays, twice in a row with different inputs, and compare each result with the context
path's tdagw_apply(LOWRANK) at the tolerance of the other apply tests.  This file is
collected last so a failure here leaves every other test already run.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2502_05635_gb300 as tg  # noqa: E402


def _c64(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.complex64).cuda()


@pytest.mark.parametrize("L,nc,rank", [(12, 1, 29), (9, 2, 64), (24, 1, 256)])
def test_noalloc_matches_context_apply_twice(L, nc, rank):
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, rank)
    stream = torch.cuda.current_stream().cuda_stream
    ctx = tg.Context(p, tg.C64, stream=stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    ld = rank + (rank & 1)
    Up = np.zeros((mdl.N, ld), np.complex128)
    Vp = np.zeros((mdl.N, ld), np.complex128)
    Up[:, :rank], Vp[:, :rank] = U, V
    Ud, Vd, dd = _c64(Up), _c64(Vp), _c64(d)
    Sd = torch.from_numpy(S.astype(np.float32)).cuda()
    for seed in (11, 12):                       # two calls in a row, different inputs
        x = _c64(wl.random_state(mdl.N, seed))
        y_ref = torch.empty_like(x)
        y = torch.empty_like(x)
        tg.tdagw_apply(ctx.h, tg.LOWRANK, x, y_ref)
        tg.tdagw_apply_lowrank_noalloc(Ud, Vd, Sd, dd, x, y, stream)
        torch.cuda.synchronize()
        ref = y_ref.cpu().numpy()
        err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < 2e-6, (seed, err)
    ctx.close()


def test_noalloc_small_N_wide_ld_vs_numpy():
    """N below the 152 row blocks of the V^H x pass (one block per row) and a row stride
    far above the rank, against a NumPy complex128 evaluation of diag o x + U (S o (V^H x))."""
    N, rank, ld = 64, 24, 40
    rng = np.random.default_rng(21)
    U = (rng.standard_normal((N, ld)) + 1j * rng.standard_normal((N, ld))) / 20
    V = (rng.standard_normal((N, ld)) + 1j * rng.standard_normal((N, ld))) / 20
    S = rng.uniform(0.1, 1.0, rank).astype(np.float32)
    d = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Ud, Vd, dd = _c64(U), _c64(V), _c64(d)
    Sd = torch.from_numpy(S).cuda()
    # the padding columns [rank, ld) hold values that must not enter the result
    for seed in (31, 32):
        xh = wl.random_state(N, seed)
        x = _c64(xh)
        y = torch.empty_like(x)
        tg.tdagw_apply_lowrank_noalloc(Ud, Vd, Sd, dd, x, y)
        torch.cuda.synchronize()
        Uc, Vc = U.astype(np.complex64).astype(complex), V.astype(np.complex64).astype(complex)
        xc = xh.astype(np.complex64).astype(complex)
        want = d.astype(np.complex64) * xc + Uc[:, :rank] @ (S * (Vc[:, :rank].conj().T @ xc))
        err = np.abs(y.cpu().numpy() - want).max() / np.abs(want).max()
        assert err < 2e-6, (seed, err)


def test_noalloc_rejects_host_pointers():
    """Host memory passed where device memory is expected is refused before any launch."""
    import ctypes as ct
    N, rank = 64, 8
    Ud = torch.zeros((N, rank), dtype=torch.complex64, device="cuda")
    Sd = torch.ones(rank, dtype=torch.float32, device="cuda")
    dd = torch.zeros(N, dtype=torch.complex64, device="cuda")
    y = torch.zeros(N, dtype=torch.complex64, device="cuda")
    xh = np.zeros(N, np.complex64)
    rc = tg.lib().tdagw_apply_lowrank_noalloc(
        ct.c_void_p(Ud.data_ptr()), ct.c_void_p(Ud.data_ptr()), rank, ct.c_void_p(Sd.data_ptr()),
        ct.c_void_p(dd.data_ptr()), N, rank, ct.c_void_p(xh.ctypes.data), ct.c_void_p(y.data_ptr()), None)
    assert rc == tg.ERR_INVALID_ARG and "x" in tg.tdagw_last_error()


def test_noalloc_takes_no_device_memory_after_first_call():
    N, rank = 1296, 64
    rng = np.random.default_rng(3)
    Ud = _c64(rng.standard_normal((N, rank)) / 40)
    Vd = _c64(rng.standard_normal((N, rank)) / 40)
    Sd = torch.ones(rank, dtype=torch.float32, device="cuda")
    dd = _c64(np.full(N, -0.01))
    x = _c64(wl.random_state(N, 5))
    y = torch.empty_like(x)
    tg.tdagw_apply_lowrank_noalloc(Ud, Vd, Sd, dd, x, y)
    torch.cuda.synchronize()
    # device-wide free memory (sees any cudaMalloc of the library, which torch's own
    # counters would not) and torch's allocator, which this process alone uses
    alloc0 = torch.cuda.memory_allocated()
    free0 = torch.cuda.mem_get_info()[0]
    for _ in range(3):
        tg.tdagw_apply_lowrank_noalloc(Ud, Vd, Sd, dd, x, y)
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.mem_get_info()[0] >= free0


def test_noalloc_rejects_bad_sizes():
    N = 64
    Ud = torch.zeros((N, 2050), dtype=torch.complex64, device="cuda")
    Sd = torch.ones(2049, dtype=torch.float32, device="cuda")
    dd = torch.zeros(N, dtype=torch.complex64, device="cuda")
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    y = torch.zeros_like(x)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_apply_lowrank_noalloc(Ud, Ud, Sd, dd, x, y)
    assert e.value.code == tg.ERR_INVALID_ARG and "2048" in str(e.value)
    Uo = torch.zeros((N, 7), dtype=torch.complex64, device="cuda")
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_apply_lowrank_noalloc(Uo, Uo, Sd[:7], dd, x, y)
    assert e.value.code == tg.ERR_INVALID_ARG
