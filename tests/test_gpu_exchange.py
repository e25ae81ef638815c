"""Direct + exchange kernel (Eq. bse-exchange-def for the lattice model) and the k-block
reading of K^diag on the GPU, through the C ABI, vs the FP64 oracle.  Same factors on both
sides for the low-rank parity; the GPU's randomised SVD of the k-block split against the
oracle's Eckart-Young optimum."""
import dataclasses

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


def _ctx(p, dtype):
    return tg.Context(p, dtype, stream=torch.cuda.current_stream().cuda_stream)


def _tensor(x, dtype):
    t = torch.from_numpy(np.ascontiguousarray(x))
    return (t.to(torch.complex64) if dtype == tg.C64 else t).cuda()


GRIDS = [(5, 2, 1.0), (12, 1, 0.5), (9, 2, 2.0)]   # L, copies, lambda_x: N = 400, 576, 1296


@pytest.fixture(scope="module", params=GRIDS, ids=lambda g: f"L{g[0]}nb{2 * g[1]}x{g[2]}")
def grid(request):
    L, nc, lx = request.param
    p = dataclasses.replace(wl.small_model(L, nc), exchange=lx)
    mdl = om.Model(p)
    return p, mdl, ok.dense_kernel(mdl)


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_kernel_with_exchange_entries_and_apply(grid, dtype):
    p, mdl, K = grid
    c = _ctx(p, dtype)
    rng = np.random.default_rng(1)
    r = np.concatenate([rng.integers(0, mdl.N, 4000), np.arange(mdl.N)])
    cc = np.concatenate([rng.integers(0, mdl.N, 4000), np.arange(mdl.N)])
    got = tg.tdagw_get_kernel_entries(c.h, r, cc)
    tol = 1e-13 if dtype == tg.C128 else 2e-7
    assert np.abs(got - K[r, cc]).max() <= tol * np.abs(K).max()
    x = wl.random_state(mdl.N, 2)
    y = torch.empty(mdl.N, dtype=torch.complex64 if dtype == tg.C64 else torch.complex128, device="cuda")
    tg.tdagw_apply(c.h, tg.FULL, _tensor(x, dtype), y)
    torch.cuda.synchronize()
    ref = K @ x
    assert np.abs(y.cpu().numpy() - ref).max() <= (1e-12 if dtype == tg.C128 else 2e-6) * np.abs(ref).max()


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_kblock_lowrank_apply_vs_oracle(grid, dtype):
    p, mdl, K = grid
    B, Koff = ok.split_kblocks(K, p.Nb)
    U, S, V = olr.truncated_svd(Koff, 17)
    c = _ctx(p, dtype)
    tg.tdagw_set_kdiag_blocks(c.h, True)
    x = wl.random_state(mdl.N, 3)
    ref = olr.apply_lowrank_kblocks(B, U, S, V, x)
    tol = 1e-12 if dtype == tg.C128 else 2e-6
    for blocks in (B, None):   # blocks from the host, or from the device kernel
        tg.tdagw_set_factors(c.h, U, S, V, blocks)
        y = torch.empty(mdl.N, dtype=torch.complex64 if dtype == tg.C64 else torch.complex128, device="cuda")
        tg.tdagw_apply(c.h, tg.LOWRANK, _tensor(x, dtype), y)
        torch.cuda.synchronize()
        assert np.abs(y.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()
    U2, S2, V2, B2 = tg.tdagw_get_factors(c.h, kblocks=True)
    # the last blocks came from the device kernel: independent FP64 evaluations of the
    # eigenvectors and W0 agree to ~1e-14 (c128), the stored c64 values to FP32 rounding
    assert np.abs(B2 - B).max() <= (1e-13 if dtype == tg.C128 else 2e-7) * np.abs(B).max()


@pytest.mark.parametrize("dtype,flags,tol", [(tg.C64, tg.FLAG_RESET, 1e-5),
                                             (tg.C64, tg.FLAG_RESET | tg.FLAG_STAGEWISE, 1e-5),
                                             (tg.C128, tg.FLAG_RESET, 1e-10)],
                         ids=["c64-persistent", "c64-stagewise", "c128"])
def test_kblock_propagation_vs_oracle(grid, dtype, flags, tol):
    p, mdl, K = grid
    B, Koff = ok.split_kblocks(K, p.Nb)
    U, S, V = olr.truncated_svd(Koff, 23)
    c = _ctx(p, dtype)
    tg.tdagw_set_kdiag_blocks(c.h, True)
    tg.tdagw_set_factors(c.h, U, S, V, B)
    pulse = wl.Pulse(E0=4e-3, omega=0.12, t0=10.0, sigma=5.0)
    T = 150
    s = op.half_step_samples(pulse, 0.2, T)
    ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank_kblocks(B, U, S, V, v), s, 0.2, T)
    got = c.propagate(pulse, T, 0.2, tg.LOWRANK, flags=flags)
    assert np.abs(ref[:, 0]).max() > 1e-8
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < tol, j


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_kblock_rsvd_near_optimal(dtype):
    """The GPU's randomised SVD of K minus its k = k' blocks (direct + exchange kernel)."""
    p = dataclasses.replace(wl.small_model(12, 1), exchange=1.0)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    B, Koff = ok.split_kblocks(K, p.Nb)
    sv = olr.singular_values(Koff)
    c = _ctx(p, dtype)
    tg.tdagw_set_kdiag_blocks(c.h, True)
    r = 29
    tg.tdagw_compress_svd(c.h, r, 64, 2, 1)
    U, S, V, B2 = tg.tdagw_get_factors(c.h, kblocks=True)
    err = np.linalg.norm(Koff - (U * S) @ V.conj().T)
    opt = np.sqrt(np.sum(sv[r:] ** 2))
    assert err <= 1.001 * opt + 1e-6 * np.linalg.norm(Koff)
    np.testing.assert_allclose(S[:4], sv[:4], rtol=1e-6 if dtype == tg.C64 else 1e-8)
    assert np.abs(B2 - B).max() <= 2e-7 * np.abs(B).max()


def test_kblock_mode_errors_and_reset():
    p = wl.small_model(4, 1)
    c = _ctx(p, tg.C64)
    q = wl.Pulse()
    tg.tdagw_compress_svd(c.h, 5, 8, 1, 1)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_set_kdiag_blocks(c.h, 2)
    assert e.value.code == tg.ERR_INVALID_ARG
    tg.tdagw_set_kdiag_blocks(c.h, True)   # the strict-diagonal factors are removed
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(c.h, [tg.make_field(q)], [5], 0.2, tg.LOWRANK)
    assert e.value.code == tg.ERR_NO_FACTORS
    tg.tdagw_compress_svd(c.h, 5, 8, 1, 1)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(c.h, [tg.make_field(q)] * 2, [5] * 2, 0.2, tg.LOWRANK,
                           tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    assert e.value.code == tg.ERR_UNSUPPORTED
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_compress_svd(c.h, 5, 8, 1, 1, precision=1)
    assert e.value.code == tg.ERR_UNSUPPORTED
    tg.tdagw_set_kdiag_blocks(c.h, False)
    tg.tdagw_compress_svd(c.h, 5, 8, 1, 1)
    c.propagate(q, 5, 0.2, tg.LOWRANK)


def _kblock_case(L, nc, lx, rank):
    p = dataclasses.replace(wl.small_model(L, nc), exchange=lx)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    B, Koff = ok.split_kblocks(K, p.Nb)
    U, S, V = olr.truncated_svd(Koff, rank)
    apply = lambda v: olr.apply_lowrank_kblocks(B, U, S, V, v)  # noqa: E731
    BH = np.conj(np.swapaxes(B, 1, 2))
    applyH = lambda v: (np.einsum("kpq,kq->kp", BH, v.reshape(B.shape[0], B.shape[1])).reshape(-1)  # noqa: E731
                        + V @ (S * (U.conj().T @ v)))
    return p, mdl, B, U, S, V, apply, applyH


@pytest.mark.parametrize("L,nc,lx,rank", [(5, 2, 1.0, 19), (12, 1, 0.5, 29)])
def test_kblock_batched_vs_oracle(L, nc, lx, rank):
    """The batched FP32 path with the k-block term: four trajectories of uneven length in
    one launch, each against the oracle with the same factors and blocks."""
    p, mdl, B, U, S, V, apply, _ = _kblock_case(L, nc, lx, rank)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_kdiag_blocks(c.h, True)
    tg.tdagw_set_factors(c.h, U, S, V, B)
    pulses = [wl.Pulse(E0=4e-3, omega=0.12, t0=8.0, sigma=4.0),
              wl.Pulse(E0=2e-3, omega=0.09, t0=6.0, sigma=3.0, dir_x=0.6, dir_y=0.8),
              wl.Pulse(E0=6e-3, omega=0.14, t0=5.0, sigma=2.0),
              wl.Pulse(E0=1e-3, omega=0.11, t0=7.0, sigma=5.0, dir_x=0.0, dir_y=1.0)]
    steps = [90, 37, 90, 61]
    got = c.propagate_batch(pulses, steps, 0.2, tg.LOWRANK)
    for b, (q, T) in enumerate(zip(pulses, steps)):
        s = op.half_step_samples(q, 0.2, T)
        ref, _ = op.rk4(mdl, apply, s, 0.2, T, direction=(q.dir_x, q.dir_y))
        for j in range(3):
            assert op.rel_l2(got[:T + 1, b, j], ref[:, j]) < 1e-5, (b, j)
        assert np.all(np.isnan(got[T + 1:, b]))


@pytest.mark.parametrize("L,nc,lx,rank", [(4, 1, 1.0, 9), (3, 2, 1.0, 20)])
def test_kblock_adjoint_vs_oracle(L, nc, lx, rank):
    """The discrete adjoint with the k-block term (K^H applies the conjugate-transposed
    blocks) against the oracle adjoint: field-sample and pulse-parameter gradients."""
    from oracle import adjoint as oa
    p, mdl, B, U, S, V, apply, applyH = _kblock_case(L, nc, lx, rank)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_kdiag_blocks(c.h, True)
    tg.tdagw_set_factors(c.h, U, S, V, B)
    pulses = [wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0),
              wl.Pulse(E0=0.015, omega=0.11, t0=4.0, sigma=2.5, dir_x=0.6, dir_y=0.8)]
    dt, steps = 0.2, [60, 45]
    tg.tdagw_propagate(c.h, [tg.make_field(q) for q in pulses], steps, dt, tg.LOWRANK,
                       tg.FLAG_RESET | tg.FLAG_CHECKPOINT)
    dJ = np.zeros((61, 2, 3))
    refs = []
    for b, (q, T) in enumerate(zip(pulses, steps)):
        s = op.half_step_samples(q, dt, T)
        obs, _ = op.rk4(mdl, apply, s, dt, T, direction=(q.dir_x, q.dir_y))
        _, dJdP = oa.spectral_objective(obs[:, 0], dt, q.omega)
        dJ[:T + 1, b, 0] = dJdP
        gE = oa.adjoint(mdl, apply, applyH, s, dt, T, (q.dir_x, q.dir_y), dJdP)
        refs.append((gE, oa.pulse_param_jacobian(q, dt, T).T @ gE))
    gE_gpu, gp_gpu = tg.tdagw_adjoint(c.h, dJ, 60, 2)
    for b, (T, (gE, gp)) in enumerate(zip(steps, refs)):
        assert np.linalg.norm(gE_gpu[:2 * T + 1, b] - gE) / np.linalg.norm(gE) < 1e-4, b
        np.testing.assert_allclose(gp_gpu[b], gp, rtol=1e-4, atol=1e-4 * np.abs(gp).max())
