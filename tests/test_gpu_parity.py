"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Small grids span several GEMV tiles and a ragged tail (N = 400, 576, 1296, 2304); the
full mos2-size grid (N = 20736) is checked on sampled entries, sampled rows, and on a
propagation prefix against the oracle's FFT form of K.x (pinned to the dense K on small
grids).  Tolerances: c128 path 1e-10 (rounding only), c64 path 1e-5 relative L2 on P(t)
(the FP32 bar of the method), applies 2e-6 relative max error (FP32 GEMV of N terms).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om
from oracle import propagate as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2502_05635_gb300 as tg  # noqa: E402


def _stream():
    return torch.cuda.current_stream().cuda_stream


def _ctx(p, dtype):
    return tg.Context(p, dtype, stream=_stream())


def _tensor(x, dtype):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return (t.to(torch.complex64) if dtype == tg.C64 else t).cuda()


GRIDS = [(5, 2), (12, 1), (9, 2), (24, 1)]   # N = 400, 576, 1296, 2304


@pytest.fixture(scope="module", params=GRIDS, ids=lambda g: f"L{g[0]}nb{2 * g[1]}")
def grid(request):
    L, nc = request.param
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    return p, mdl, ok.dense_kernel(mdl)


# ---------------------------------------------------------------- model + kernel -------

def test_model_matches_oracle(grid):
    p, mdl, _ = grid
    c = _ctx(p, tg.C128)
    m = tg.tdagw_get_model(c.h)
    np.testing.assert_allclose(m["eps"], mdl.eps, atol=1e-14)
    np.testing.assert_allclose(m["U"], mdl.U, atol=1e-14)
    for key, ref in (("dx", mdl.dx), ("dy", mdl.dy), ("vx", mdl.vx)):
        np.testing.assert_allclose(m[key], ref, atol=1e-9, err_msg=key)


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_kernel_entries(grid, dtype):
    p, mdl, K = grid
    c = _ctx(p, dtype)
    rng = np.random.default_rng(1)
    r = rng.integers(0, mdl.N, 4000)
    cc = rng.integers(0, mdl.N, 4000)
    r = np.concatenate([r, np.arange(mdl.N)])          # the whole diagonal too
    cc = np.concatenate([cc, np.arange(mdl.N)])
    got = tg.tdagw_get_kernel_entries(c.h, r, cc)
    # independent FP64 evaluations (quadrature of W0, eigenvectors) agree to ~1e-14
    tol = 1e-13 if dtype == tg.C128 else 2e-7
    assert np.abs(got - K[r, cc]).max() <= tol * np.abs(K).max()


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_apply_full(grid, dtype):
    p, mdl, K = grid
    c = _ctx(p, dtype)
    x = wl.random_state(mdl.N, 9)
    y = torch.empty_like(_tensor(x, dtype))
    tg.tdagw_apply(c.h, tg.FULL, _tensor(x, dtype), y)
    torch.cuda.synchronize()
    ref = K @ x
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if dtype == tg.C128 else 2e-6), err


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
@pytest.mark.parametrize("rank", [1, 7, 64])
def test_apply_lowrank(grid, dtype, rank):
    p, mdl, K = grid
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, rank)
    c = _ctx(p, dtype)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    x = wl.random_state(mdl.N, 4)
    y = torch.empty_like(_tensor(x, dtype))
    tg.tdagw_apply(c.h, tg.LOWRANK, _tensor(x, dtype), y)
    torch.cuda.synchronize()
    ref = olr.apply_lowrank(d, U, S, V, x)
    err = np.abs(y.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < (1e-13 if dtype == tg.C128 else 2e-6), err
    U2, S2, V2, d2 = tg.tdagw_get_factors(c.h)
    tol = 1e-15 if dtype == tg.C128 else 1e-7
    assert np.abs(U2 - U).max() < tol and np.abs(V2 - V).max() < tol
    assert np.abs(S2 - S).max() < tol * S.max()


# ---------------------------------------------------------------- propagation ----------

@pytest.fixture(scope="module")
def cfg0():
    w = wl.tiny_nb2_l12()
    mdl = om.Model(w.model)
    K = ok.dense_kernel(mdl)
    s = op.half_step_samples(w.pulses[0], w.dt, w.steps[0])
    ref, xT = op.rk4(mdl, lambda v: K @ v, s, w.dt, w.steps[0])
    return w, mdl, K, ref, xT


@pytest.mark.parametrize("dtype,tol", [(tg.C128, 1e-10), (tg.C64, 1e-5)])
def test_propagate_full_cfg0(cfg0, dtype, tol):
    """The 2000-step, 12 x 12 two-band trajectory: P, J, occupation vs the oracle."""
    w, mdl, K, ref, xT = cfg0
    c = _ctx(w.model, dtype)
    got = c.propagate(w.pulses[0], w.steps[0], w.dt, tg.FULL)
    assert got.shape == ref.shape
    for j in range(3):
        e = op.rel_l2(got[:, j], ref[:, j])
        assert e < tol, (j, e)
    drho, _, step = tg.tdagw_get_state(c.h)
    assert step == w.steps[0]
    assert np.abs(drho - xT).max() < tol * 10 * np.abs(xT).max()


@pytest.mark.parametrize("dtype,tol", [(tg.C128, 1e-10), (tg.C64, 1e-5)])
def test_propagate_lowrank_cfg0(cfg0, dtype, tol):
    """Low-rank path with the oracle's exact factors at 5% rank, same factors both sides."""
    w, mdl, K, _, _ = cfg0
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 29)
    s = op.half_step_samples(w.pulses[0], w.dt, w.steps[0])
    ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, w.dt, w.steps[0])
    c = _ctx(w.model, dtype)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    got = c.propagate(w.pulses[0], w.steps[0], w.dt, tg.LOWRANK)
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < tol


@pytest.mark.parametrize("L,nc,rank", [(5, 2, 7), (12, 1, 1), (9, 2, 64), (24, 1, 256)])
def test_persistent_lowrank_vs_oracle_and_stagewise(L, nc, rank):
    """Single-launch persistent low-rank kernel (c64) on grids with ragged per-CTA row
    ranges and odd ranks: vs the oracle with the same factors, and vs the stage-wise
    kernels (different summation order only)."""
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, rank)
    pulse = wl.Pulse(E0=2e-3, omega=0.1, t0=20.0, sigma=8.0)
    T = 250
    s = op.half_step_samples(pulse, 0.2, T)
    ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, 0.2, T)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    a = c.propagate(pulse, T, 0.2, tg.LOWRANK)
    b = c.propagate(pulse, T, 0.2, tg.LOWRANK, flags=tg.FLAG_RESET | tg.FLAG_STAGEWISE)
    for j in range(3):
        assert op.rel_l2(a[:, j], ref[:, j]) < 1e-5, j
        assert op.rel_l2(a[:, j], b[:, j]) < 1e-6, j


@pytest.mark.parametrize("L,nc,rank,kblocks", [(13, 1, 40, False), (14, 2, 64, False), (14, 2, 33, True),
                                                (40, 1, 128, True)])
def test_persistent_uneven_shares_vs_oracle(L, nc, rank, kblocks):
    """More k-points than CTAs (169, 196 and 1600 k-points over at most 152 CTAs: CTAs own
    one or two more k-points than others), with and without the k = k' block term.  Seeded
    factors (and seeded Hermitian blocks) on both sides; vs the oracle and vs the
    stage-wise kernels."""
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, rank, seed=L + rank)
    P = mdl.Nb * mdl.Nb
    if kblocks:
        rng = np.random.default_rng(L)
        Bk = 0.004 * (rng.standard_normal((mdl.Nk, P, P)) + 1j * rng.standard_normal((mdl.Nk, P, P)))
        Bk = Bk + np.conj(np.swapaxes(Bk, 1, 2))
        apply = lambda v: olr.apply_lowrank_kblocks(Bk, U, S, V, v)  # noqa: E731
    else:
        apply = lambda v: olr.apply_lowrank(d, U, S, V, v)  # noqa: E731
    pulse = wl.Pulse(E0=3e-3, omega=0.1, t0=10.0, sigma=4.0)
    T = 120
    ref, _ = op.rk4(mdl, apply, op.half_step_samples(pulse, 0.2, T), 0.2, T)
    c = _ctx(p, tg.C64)
    if kblocks:
        tg.tdagw_set_kdiag_blocks(c.h, True)
        tg.tdagw_set_factors(c.h, U, S, V, Bk)
    else:
        tg.tdagw_set_factors(c.h, U, S, V, d)
    a = c.propagate(pulse, T, 0.2, tg.LOWRANK)
    b = c.propagate(pulse, T, 0.2, tg.LOWRANK, flags=tg.FLAG_RESET | tg.FLAG_STAGEWISE)
    assert np.abs(ref[:, 0]).max() > 1e-7
    for j in range(3):
        assert op.rel_l2(a[:, j], ref[:, j]) < 1e-5, j
        assert op.rel_l2(a[:, j], b[:, j]) < 1e-6, j


def test_persistent_timeout_is_reported_and_context_survives(cfg0):
    """Fault injection on the host side of a bounded wait: the grid barrier waits for a
    block that does not exist; every wait gives up after its budget, the call reports
    TDAGW_ERR_TIMEOUT, and the same context then propagates normally."""
    w = cfg0[0]
    c = _ctx(w.model, tg.C64)
    d, Koff = ok.split_diag_off(cfg0[2])
    U, S, V = olr.truncated_svd(Koff, 29)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    tg.tdagw_propagate(c.h, [tg.make_field(w.pulses[0])], [50], w.dt, tg.LOWRANK,
                       tg.FLAG_RESET | tg.FLAG_TEST_TIMEOUT)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_sync(c.h)
    assert e.value.code == tg.ERR_TIMEOUT
    good = c.propagate(w.pulses[0], 50, w.dt, tg.LOWRANK)
    ref = c.propagate(w.pulses[0], 50, w.dt, tg.LOWRANK, flags=tg.FLAG_RESET | tg.FLAG_STAGEWISE)
    assert op.rel_l2(good[:, 0], ref[:, 0]) < 1e-6


def test_graph_and_stagewise_launches_agree(cfg0):
    w = cfg0[0]
    c = _ctx(w.model, tg.C64)
    a = c.propagate(w.pulses[0], 300, w.dt, tg.FULL)
    b = c.propagate(w.pulses[0], 300, w.dt, tg.FULL, flags=tg.FLAG_RESET | tg.FLAG_NO_GRAPH)
    assert np.array_equal(a, b)


def test_resume_is_bitwise(cfg0):
    """get_state / set_state between two halves reproduces the uninterrupted run exactly."""
    w = cfg0[0]
    c = _ctx(w.model, tg.C64)
    full = c.propagate(w.pulses[0], 400, w.dt, tg.FULL)
    first = c.propagate(w.pulses[0], 170, w.dt, tg.FULL)
    drho, carry, step = tg.tdagw_get_state(c.h)
    c2 = _ctx(w.model, tg.C64)
    tg.tdagw_set_state(c2.h, drho, carry, step)
    second = c2.propagate(w.pulses[0], 230, w.dt, tg.FULL, flags=0)
    assert np.array_equal(first, full[:171])
    assert np.array_equal(second, full[170:])


def test_kahan_reduces_accumulation_error(cfg0):
    """10000 steps: the compensated FP32 state stays within the FP32 bar and no worse than
    the plain accumulation, whose per-step rounding grows as a random walk."""
    w, mdl, K = cfg0[:3]
    T = 10000
    ref, _ = op.rk4(mdl, lambda v: K @ v, op.half_step_samples(w.pulses[0], w.dt, T), w.dt, T)
    c = _ctx(w.model, tg.C64)
    e_k = op.rel_l2(c.propagate(w.pulses[0], T, w.dt, tg.FULL)[:, 0], ref[:, 0])
    e_p = op.rel_l2(c.propagate(w.pulses[0], T, w.dt, tg.FULL,
                                flags=tg.FLAG_RESET | tg.FLAG_NO_KAHAN)[:, 0], ref[:, 0])
    print(f"10000 steps: compensated {e_k:.3e}, plain {e_p:.3e}")
    assert e_k < 1e-5
    assert e_k <= 1.05 * e_p


def test_zero_steps_and_zero_field():
    p = wl.small_model(4, 2)
    c = _ctx(p, tg.C64)
    o = c.propagate(wl.Pulse(), 0, 0.2, tg.FULL)
    assert o.shape == (1, 3) and np.all(o == 0)
    o = c.propagate(wl.Pulse(E0=0.0), 50, 0.2, tg.FULL)
    assert np.all(o == 0)


def test_single_k_rabi_closed_form():
    """Nk = 1 under a constant field: the GPU c128 path meets the closed form to O(dt^4)."""
    import scipy.linalg
    p = wl.small_model(1, 1)
    mdl = om.Model(p)
    c = _ctx(p, tg.C128)
    E, dt, T = 0.01, 0.1, 400
    c.propagate(wl.Pulse(E0=E, kind=1), T, dt, tg.FULL)
    drho, _, _ = tg.tdagw_get_state(c.h)
    W0 = -ok.dense_kernel(mdl)[0, 0].real
    rho0 = mdl.rho0()[0]
    Ut = scipy.linalg.expm(-1j * (np.diag(mdl.eps[0]) + E * mdl.dx[0] + W0 * rho0) * (T * dt))
    exact = Ut @ rho0 @ Ut.conj().T
    assert np.abs(rho0 + drho.reshape(2, 2) - exact).max() < 1e-7


def test_table_field_matches_analytic(cfg0):
    w = cfg0[0]
    c = _ctx(w.model, tg.C64)
    a = c.propagate(w.pulses[0], 200, w.dt, tg.FULL)
    tab = op.half_step_samples(w.pulses[0], w.dt, 200)
    b = c.propagate(w.pulses[0], 200, w.dt, tg.FULL, table=tab)
    assert op.rel_l2(b[:, 0], a[:, 0]) < 1e-6


def test_error_codes_on_device():
    p = wl.small_model(4, 1)
    c = _ctx(p, tg.C64)
    with pytest.raises(tg.TdagwError) as e:
        c.propagate(wl.Pulse(), 10, 0.2, tg.LOWRANK)
    assert e.value.code == tg.ERR_NO_FACTORS
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_compress_svd(c.h, 10, 64, 2)     # rank + oversample > N = 64
    assert e.value.code == tg.ERR_INVALID_ARG
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_get_kernel_entries(c.h, [0], [10 ** 9])
    assert e.value.code == tg.ERR_INVALID_ARG
    h = tg.tdagw_create(tg.model_desc(p), _stream())
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(h, [tg.make_field(wl.Pulse())], [5], 0.2, tg.FULL)
    assert e.value.code == tg.ERR_NOT_BUILT
    tg.tdagw_destroy(h)


# ---------------------------------------------------------------- randomised SVD -------

@pytest.mark.parametrize("L,rank", [(24, 256), (36, 512)])
def test_rsvd_near_optimal_at_sweep_and_gradient_sizes(L, rank):
    """The randomised SVD (p = 64, q = 2) at the field-sweep size (two-band 24 x 24, N = 2304,
    rank 256) and the differentiation size (36 x 36, N = 5184, rank 512): its truncation
    error against the Eckart-Young optimum from an exact LAPACK eigendecomposition of the
    oracle's K^off (Hermitian: sigma = |lambda|), and the leading singular values."""
    import scipy.linalg
    p = wl.small_model(L, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    del K
    lam = scipy.linalg.eigvalsh(Koff)
    sv = np.sort(np.abs(lam))[::-1]
    c = _ctx(p, tg.C64)
    tg.tdagw_compress_svd(c.h, rank, 64, 2, 1)
    U, S, V, d2 = tg.tdagw_get_factors(c.h)
    err = np.linalg.norm(Koff - (U * S) @ V.conj().T)
    opt = np.sqrt(np.sum(sv[rank:] ** 2))
    print(f"N = {mdl.N}, rank {rank}: error / optimal = {err / opt:.5f}")
    assert err <= 1.01 * opt          # HMT one-sided projection, q = 2 (the bar is 1.1)
    np.testing.assert_allclose(S[:rank // 4], sv[:rank // 4], rtol=1e-3)
    c.close()


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_rsvd_near_optimal(dtype):
    """GPU randomised SVD (p = 64, q = 2): singular values and truncation error vs LAPACK."""
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    sv = olr.singular_values(Koff)
    c = _ctx(p, dtype)
    r = 29
    tg.tdagw_compress_svd(c.h, r, 64, 2, 1)
    U, S, V, d2 = tg.tdagw_get_factors(c.h)
    err = np.linalg.norm(Koff - (U * S) @ V.conj().T)
    opt = np.sqrt(np.sum(sv[r:] ** 2))
    assert err <= 1.001 * opt + 1e-6 * np.linalg.norm(Koff)
    # two power iterations resolve the degenerate clusters of this lattice kernel to
    # ~5e-5 (the same for a numpy emulation of the scheme); the top cluster to 1e-8
    np.testing.assert_allclose(S, sv[:r], rtol=2e-4)
    np.testing.assert_allclose(S[:4], sv[:4], rtol=1e-6 if dtype == tg.C64 else 1e-8)
    np.testing.assert_allclose(np.abs(d2), np.abs(d), rtol=1e-6)
    np.testing.assert_allclose(np.abs(U.conj().T @ U), np.eye(r), atol=1e-5 if dtype == tg.C64 else 1e-12)


def test_rsvd_propagation_within_truncation_error(cfg0):
    """err(GPU low-rank vs oracle full) <= 1.1 err(oracle exact-SVD low-rank vs full) + 1e-5."""
    w, mdl, K, ref, _ = cfg0
    d, Koff = ok.split_diag_off(K)
    r = 29
    U, S, V = olr.truncated_svd(Koff, r)
    s = op.half_step_samples(w.pulses[0], w.dt, w.steps[0])
    lr, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, w.dt, w.steps[0])
    e_opt = op.rel_l2(lr[:, 0], ref[:, 0])
    c = _ctx(w.model, tg.C64)
    tg.tdagw_compress_svd(c.h, r, 64, 2, 1)
    got = c.propagate(w.pulses[0], w.steps[0], w.dt, tg.LOWRANK)
    assert op.rel_l2(got[:, 0], ref[:, 0]) <= 1.1 * e_opt + 1e-5


# ---------------------------------------------------------------- full size ------------

@pytest.fixture(scope="module")
def big():
    w = wl.mos2size_nb4_l36()
    mdl = om.Model(w.model)
    c = _ctx(w.model, tg.C64)
    return w, mdl, c


def test_full_size_kernel_and_apply_rows(big):
    w, mdl, c = big
    rng = np.random.default_rng(5)
    rows = rng.integers(0, mdl.N, 24)
    for r in rows:
        cols = rng.integers(0, mdl.N, 64)
        got = tg.tdagw_get_kernel_entries(c.h, np.full(64, r), cols)
        ref = ok.kernel_row(mdl, int(r))[cols]
        assert np.abs(got - ref).max() <= 2e-7 * np.abs(ref).max() + 1e-12
    x = wl.random_state(mdl.N, 2)
    y = torch.empty(mdl.N, dtype=torch.complex64, device="cuda")
    xt = _tensor(x, tg.C64)
    tg.tdagw_apply(c.h, tg.FULL, xt, y)
    torch.cuda.synchronize()
    yh = y.cpu().numpy()
    full = ok.apply_fft(mdl, x)
    assert np.abs(yh - full).max() < 2e-6 * np.abs(full).max()
    for r in rows:
        assert abs(yh[r] - ok.kernel_row(mdl, int(r)) @ x) < 2e-6 * np.abs(full).max()


def test_full_size_propagation_prefix(big):
    """N = 20736, dense 3.4 GB kernel, graph-captured path of the benchmark: 400 steps vs
    the oracle's FFT form of the same kernel."""
    w, mdl, c = big
    T = 400
    s = op.half_step_samples(w.pulses[0], w.dt, T)
    ref, _ = op.rk4(mdl, ok.fft_applier(mdl), s, w.dt, T)
    got = c.propagate(w.pulses[0], T, w.dt, tg.FULL)
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < 1e-5, j


def test_full_size_rsvd_properties(big):
    """rank-1024 randomised SVD at N = 20736: orthonormal columns of U and of V, and a
    residual on random probes (K^off x by the oracle's FFT form) well below ||K^off x||."""
    w, mdl, c = big
    tg.tdagw_compress_svd(c.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
    U, S, V, d = tg.tdagw_get_factors(c.h)
    assert np.all(np.diff(S) <= 1e-7 * S[0]) and S[-1] > 0
    rng = np.random.default_rng(3)
    idx = rng.integers(0, w.rank, 16)
    G = U[:, idx].conj().T @ U[:, idx]
    assert np.abs(G - np.eye(16)).max() < 1e-5
    GV = V[:, idx].conj().T @ V[:, idx]
    assert np.abs(GV - np.eye(16)).max() < 1e-4
    fft = ok.fft_applier(mdl)
    dK = ok.kernel_diag(mdl)
    for s_ in range(3):
        x = wl.random_state(mdl.N, 100 + s_)
        kx = fft(x) - dK * x
        lr = U @ (S * (V.conj().T @ x))
        assert np.linalg.norm(kx - lr) < 0.5 * np.linalg.norm(kx)


def test_full_size_lowrank_propagation(big):
    """Low-rank path at N = 20736, rank 1024 (the benchmark's persistent launch), seeded
    factors installed on the GPU and used by the oracle as well: 40 steps of a pulse that
    peaks inside the window (the benchmark pulse peaks at t = 200), P, J, occupation."""
    w, mdl, c = big
    U, S, V, d = wl.random_factors(mdl.N, w.rank, seed=17)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    T = 40
    pulse = wl.Pulse(E0=2e-3, omega=0.1, t0=4.0, sigma=2.0)
    s = op.half_step_samples(pulse, w.dt, T)
    ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, w.dt, T)
    got = c.propagate(pulse, T, w.dt, tg.LOWRANK)
    assert np.abs(ref[:, 0]).max() > 1e-6  # the response is not trivial
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < 1e-5, j
