"""Channel-wise kernel (Eq. svd-channel-wise) through the C ABI vs the FP64 oracle.

The CUDA path and the oracle use the same factors (installed from the oracle's exact
channel SVDs, or made on the GPU and read back).  Cases span both band counts, ranks 0
(diagonal channels only) to 9, per-channel ranks, grids with ragged per-CTA k ranges, the
persistent launch and the stage-wise kernels, and the full mos2-size grid (N = 20736) in
the launch configuration of the benchmark.  Tolerances: c128 1e-10 (rounding), c64 1e-5
relative L2 on P(t) (the FP32 bar of the method), applies 2e-6 relative max error.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import channel as oc
from oracle import kernel as ok
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


CASES = [(5, 1, 3), (12, 1, 9), (4, 2, 5), (6, 2, 0)]   # L, copies, rank: N = 100, 576, 256, 576


@pytest.fixture(scope="module", params=CASES, ids=lambda c: f"L{c[0]}nb{2 * c[1]}r{c[2]}")
def case(request):
    L, nc, rank = request.param
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    return p, mdl, K, oc.channel_svd(K, p.Nb, rank)


@pytest.mark.parametrize("dtype", [tg.C64, tg.C128])
def test_channel_apply_vs_oracle(case, dtype):
    p, mdl, K, (D, U, S, V) = case
    c = _ctx(p, dtype)
    x = wl.random_state(mdl.N, 7)
    ref = oc.apply_channel(D, U, S, V, x)
    tol = 1e-12 if dtype == tg.C128 else 2e-6
    for Din in (D, None):   # diagonal channels from the host, or from the device kernel
        tg.tdagw_set_channel_factors(c.h, U, S, V, Din)
        y = torch.empty(mdl.N, dtype=torch.complex64 if dtype == tg.C64 else torch.complex128, device="cuda")
        tg.tdagw_apply(c.h, tg.CHANNEL, _tensor(x, dtype), y)
        torch.cuda.synchronize()
        assert np.abs(y.cpu().numpy() - ref).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("dtype,flags,tol", [(tg.C64, tg.FLAG_RESET, 1e-5),
                                             (tg.C64, tg.FLAG_RESET | tg.FLAG_STAGEWISE, 1e-5),
                                             (tg.C128, tg.FLAG_RESET, 1e-10)],
                         ids=["c64-persistent", "c64-stagewise", "c128"])
def test_channel_propagation_vs_oracle(case, dtype, flags, tol):
    p, mdl, K, (D, U, S, V) = case
    c = _ctx(p, dtype)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    pulse = wl.Pulse(E0=5e-3, omega=0.12, t0=10.0, sigma=5.0, dir_x=0.8, dir_y=0.6)
    T = 150
    s = op.half_step_samples(pulse, 0.2, T)
    ref, _ = op.rk4(mdl, lambda v: oc.apply_channel(D, U, S, V, v), s, 0.2, T,
                    direction=(pulse.dir_x, pulse.dir_y))
    got = c.propagate(pulse, T, 0.2, tg.CHANNEL, flags=flags)
    assert np.abs(ref[:, 0]).max() > 1e-8
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < tol, j


def test_persistent_and_stagewise_agree_and_resume():
    """The persistent launch and the stage-wise kernels differ only in summation order; two
    calls of 60 steps continue the state like one of 120."""
    p = wl.small_model(9, 2)
    mdl = om.Model(p)
    D, U, S, V = oc.channel_svd(ok.dense_kernel(mdl), p.Nb, 7)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    pulse = wl.Pulse(E0=4e-3, omega=0.1, t0=8.0, sigma=4.0)
    a = c.propagate(pulse, 120, 0.2, tg.CHANNEL)
    b = c.propagate(pulse, 120, 0.2, tg.CHANNEL, flags=tg.FLAG_RESET | tg.FLAG_STAGEWISE)
    for j in range(3):
        assert op.rel_l2(a[:, j], b[:, j]) < 1e-6, j
    h1 = c.propagate(pulse, 60, 0.2, tg.CHANNEL)
    h2 = c.propagate(pulse, 60, 0.2, tg.CHANNEL, flags=0)
    assert op.rel_l2(np.concatenate([h1, h2[1:]])[:, 0], a[:, 0]) < 1e-6


@pytest.mark.parametrize("rank", [100, 200, 350])
def test_persistent_long_v_rows_vs_oracle(rank):
    """Two bands, Nk = 400: every input pair has three incoming channels of the given rank,
    so the V rows hold 300, 600 and 1050 columns and the persistent kernel's V pass runs
    with four, two and one warp groups (the smaller ranks of the other tests give eight or
    sixteen)."""
    p = wl.small_model(20, 1)
    mdl = om.Model(p)
    D, U, S, V = oc.channel_svd(ok.dense_kernel(mdl), p.Nb, rank)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    pulse = wl.Pulse(E0=5e-3, omega=0.12, t0=6.0, sigma=3.0, dir_x=0.6, dir_y=0.8)
    T = 60
    s = op.half_step_samples(pulse, 0.2, T)
    ref, _ = op.rk4(mdl, lambda v: oc.apply_channel(D, U, S, V, v), s, 0.2, T,
                    direction=(pulse.dir_x, pulse.dir_y))
    got = c.propagate(pulse, T, 0.2, tg.CHANNEL)
    assert np.abs(ref[:, 0]).max() > 1e-8
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < 1e-5, j


def test_per_channel_ranks_and_round_trip():
    """Each channel its own rank (including 0): the apply uses exactly the first z_pq
    triplets, and get returns what set installed (FP32 storage)."""
    p = wl.small_model(6, 2)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    P = p.Nb ** 2
    D, U, S, V = oc.channel_svd(K, p.Nb, 6)
    ranks = np.random.default_rng(2).integers(0, 7, (P, P)).astype(np.int32)
    np.fill_diagonal(ranks, 0)
    mask = np.arange(6)[None, None, :] < ranks[:, :, None]
    Ut, Vt, St = U * mask[:, :, None, :], V * mask[:, :, None, :], S * mask
    c = _ctx(p, tg.C64)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D, ranks=ranks)
    x = wl.random_state(mdl.N, 8)
    y = torch.empty(mdl.N, dtype=torch.complex64, device="cuda")
    tg.tdagw_apply(c.h, tg.CHANNEL, _tensor(x, tg.C64), y)
    torch.cuda.synchronize()
    ref = oc.apply_channel(D, Ut, St, Vt, x)
    assert np.abs(y.cpu().numpy() - ref).max() <= 2e-6 * np.abs(ref).max()
    rk, U2, S2, V2, D2 = tg.tdagw_get_channel_factors(c.h)
    np.testing.assert_array_equal(rk, ranks)
    r = U2.shape[-1]
    assert r == ranks.max()
    for a, b in ((U2, Ut[..., :r]), (V2, Vt[..., :r])):
        assert np.abs(a - b).max() <= 1e-7 * np.abs(b).max()
    assert np.abs(S2 - St[..., :r]).max() <= 1e-7 * St.max()
    assert np.abs(D2 - D).max() <= 1e-7 * np.abs(D).max()


@pytest.mark.parametrize("L,nc,rank,dtype", [(12, 1, 20, tg.C64), (12, 1, 20, tg.C128), (6, 2, 8, tg.C64)])
def test_compress_channels_near_optimal(L, nc, rank, dtype):
    """Randomised channel SVDs on the GPU: every channel within 1 % of its optimal
    truncation error (Eckart-Young), channel q -> p the conjugate transpose of p -> q,
    vanishing channels of rank 0, the diagonal channels equal to the kernel."""
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    P = p.Nb ** 2
    c = _ctx(p, dtype)
    tg.tdagw_compress_channels(c.h, rank, 64, 2, 1)
    ranks, U, S, V, D = tg.tdagw_get_channel_factors(c.h)
    slack = 1e-12 if dtype == tg.C128 else 1e-5
    for a in range(P):
        np.testing.assert_allclose(D[a], oc.channel_block(K, p.Nb, a, a), atol=2e-7 * np.abs(K).max())
        for b in range(P):
            if a == b:
                continue
            blk = oc.channel_block(K, p.Nb, a, b)
            z = ranks[a, b]
            if np.abs(blk).max() < 1e-15:
                assert z == 0
                continue
            assert z == rank
            sv = scipy.linalg.svdvals(blk)
            opt = np.sqrt(np.sum(sv[z:] ** 2))
            err = np.linalg.norm(blk - (U[a, b, :, :z] * S[a, b, :z]) @ V[a, b, :, :z].conj().T)
            assert err <= 1.01 * opt + slack * sv[0], (a, b, err / opt)
            np.testing.assert_allclose(S[a, b, :z], sv[:z], rtol=1e-5, atol=slack * sv[0])
            assert np.abs(U[b, a] - V[a, b]).max() <= 1e-12 and np.abs(S[b, a] - S[a, b]).max() <= 1e-12


def test_rank_zero_is_diagonal_channels_only():
    p = wl.small_model(8, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    c = _ctx(p, tg.C128)
    tg.tdagw_compress_channels(c.h, 0, 64, 2, 1)
    ranks, *_ = tg.tdagw_get_channel_factors(c.h)
    assert ranks.max() == 0
    P = p.Nb ** 2
    i = np.arange(mdl.N)
    Kd = np.where((i[:, None] % P) == (i[None, :] % P), K, 0)
    x = wl.random_state(mdl.N, 9)
    y = torch.empty(mdl.N, dtype=torch.complex128, device="cuda")
    tg.tdagw_apply(c.h, tg.CHANNEL, _tensor(x, tg.C128), y)
    torch.cuda.synchronize()
    ref = Kd @ x
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-12 * np.abs(ref).max()


def test_channel_timeout_is_reported_and_context_survives():
    """The persistent channel launch with a grid barrier that waits for a block that does
    not exist: every wait gives up after its budget, the call reports TDAGW_ERR_TIMEOUT and
    the context then propagates normally."""
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    D, U, S, V = oc.channel_svd(ok.dense_kernel(mdl), p.Nb, 9)
    c = _ctx(p, tg.C64)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    pulse = wl.Pulse(E0=2e-3, omega=0.1, t0=8.0, sigma=4.0)
    tg.tdagw_propagate(c.h, [tg.make_field(pulse)], [40], 0.2, tg.CHANNEL,
                       tg.FLAG_RESET | tg.FLAG_TEST_TIMEOUT)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_sync(c.h)
    assert e.value.code == tg.ERR_TIMEOUT
    a = c.propagate(pulse, 40, 0.2, tg.CHANNEL)
    b = c.propagate(pulse, 40, 0.2, tg.CHANNEL, flags=tg.FLAG_RESET | tg.FLAG_STAGEWISE)
    assert op.rel_l2(a[:, 0], b[:, 0]) < 1e-6


def test_channel_errors():
    p = wl.small_model(4, 1)
    c = _ctx(p, tg.C64)
    q = wl.Pulse()
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(c.h, [tg.make_field(q)], [5], 0.2, tg.CHANNEL)
    assert e.value.code == tg.ERR_NO_FACTORS
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_get_channel_factors(c.h)
    assert e.value.code == tg.ERR_NO_FACTORS
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_compress_channels(c.h, 17, 8, 1)
    assert e.value.code == tg.ERR_INVALID_ARG
    tg.tdagw_compress_channels(c.h, 3, 8, 1)
    for flags, B in ((tg.FLAG_RESET | tg.FLAG_CHECKPOINT, 1), (tg.FLAG_RESET | tg.FLAG_CHECKPOINT, 3),
                     (tg.FLAG_SPLIT_F16, 2), (tg.FLAG_RESET | tg.FLAG_SPLIT_F16 | tg.FLAG_CHECKPOINT, 2)):
        with pytest.raises(tg.TdagwError) as e:
            tg.tdagw_propagate(c.h, [tg.make_field(q)] * B, [5] * B, 0.2, tg.CHANNEL, flags)
        assert e.value.code == tg.ERR_UNSUPPORTED


@pytest.mark.parametrize("L,nc,rank", [(12, 1, 9), (6, 2, 5), (9, 2, 7)])
def test_channel_batched_vs_oracle(L, nc, rank):
    """B trajectories of uneven length in one batched launch with the channel-wise kernel
    (per-channel ranks, vanishing cross-copy channels for four bands): every trajectory
    against the oracle with the same factors, and against the single-trajectory path."""
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    P = p.Nb ** 2
    D, U, S, V = oc.channel_svd(ok.dense_kernel(mdl), p.Nb, rank)
    ranks = np.random.default_rng(L).integers(1, rank + 1, (P, P)).astype(np.int32)
    np.fill_diagonal(ranks, 0)
    mask = np.arange(rank)[None, None, :] < ranks[:, :, None]
    U, V, S = U * mask[:, :, None, :], V * mask[:, :, None, :], S * mask
    c = _ctx(p, tg.C64)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D, ranks=ranks)
    pulses = [wl.Pulse(E0=5e-3, omega=0.12, t0=8.0, sigma=4.0),
              wl.Pulse(E0=2e-3, omega=0.09, t0=6.0, sigma=3.0, dir_x=0.6, dir_y=0.8),
              wl.Pulse(E0=8e-3, omega=0.14, t0=5.0, sigma=2.0),
              wl.Pulse(E0=1e-3, omega=0.11, t0=7.0, sigma=5.0, dir_x=0.0, dir_y=1.0),
              wl.Pulse(E0=3e-3, omega=0.10, t0=4.0, sigma=2.5)]
    steps = [80, 23, 80, 57, 1]
    got = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL)
    apply = lambda v: oc.apply_channel(D, U, S, V, v)  # noqa: E731
    for b, (q, T) in enumerate(zip(pulses, steps)):
        s = op.half_step_samples(q, 0.2, T)
        ref, _ = op.rk4(mdl, apply, s, 0.2, T, direction=(q.dir_x, q.dir_y))
        for j in range(3):
            assert op.rel_l2(got[:T + 1, b, j], ref[:, j]) < 1e-5, (b, j)
        assert np.all(np.isnan(got[T + 1:, b]))
    one = c.propagate(pulses[0], steps[0], 0.2, tg.CHANNEL)
    assert op.rel_l2(got[:, 0, 0], one[:, 0]) < 1e-6


def test_full_size_channel_propagation():
    """N = 20736 (four bands, 36 x 36), the persistent launch of the benchmark.  (1) The GPU's
    randomised channel SVDs at rank 65 (5 % of Nk) are near the optimum on sampled channels
    (blocks from the kernel formula).  (2) With the oracle's exact channel factors installed,
    30 steps of an early pulse match the oracle's propagation with the same factors."""
    w = wl.mos2size_channel()
    mdl = om.Model(w.model)
    c = _ctx(w.model, tg.C64)
    tg.tdagw_compress_channels(c.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED)
    ranks, U, S, V, _ = tg.tdagw_get_channel_factors(c.h)
    P = w.model.Nb ** 2
    nz = [(a, b) for a in range(P) for b in range(P) if a != b and ranks[a, b] > 0]
    assert len(nz) == 48 and all(ranks[a, b] == w.rank for a, b in nz)
    for a, b in nz[::9]:
        blk = oc.channel_block_from_model(mdl, a, b)
        sv = scipy.linalg.svdvals(blk)
        opt = np.sqrt(np.sum(sv[w.rank:] ** 2))
        z = w.rank
        err = np.linalg.norm(blk - (U[a, b, :, :z] * S[a, b, :z]) @ V[a, b, :, :z].conj().T)
        assert err <= 1.01 * opt + 1e-6 * sv[0], (a, b, err / opt)
    del U, S, V
    D, U, S, V = oc.channel_svd_from_model(mdl, w.rank)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    T = 30
    pulse = wl.Pulse(E0=2e-3, omega=0.1, t0=3.0, sigma=1.5)
    s = op.half_step_samples(pulse, w.dt, T)
    ref, _ = op.rk4(mdl, lambda v: oc.apply_channel(D, U, S, V, v), s, w.dt, T)
    got = c.propagate(pulse, T, w.dt, tg.CHANNEL)
    assert np.abs(ref[:, 0]).max() > 1e-7
    for j in range(3):
        assert op.rel_l2(got[:, j], ref[:, j]) < 1e-5, j
