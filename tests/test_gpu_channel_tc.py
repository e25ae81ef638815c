"""Channel-wise kernel (Eq. svd-channel-wise) with split-FP16 segment tiles on the tensor
cores (TDAGW_FLAG_SPLIT_F16 with mode CHANNEL) through the C ABI vs the FP64 oracle.

Both sides use the same channel factors (the oracle's exact channel SVDs, installed with
tdagw_set_channel_factors).  Cases: both band counts; k-point counts that are not a
multiple of the 16-row chunk or the 256-row tile; per-channel ranks including zero; only
the dense diagonal channels (rank 0); long V rows (several 256-column tiles per segment);
more trajectories than one 64-trajectory group; uneven lengths including a zero-step
trajectory; the mos2-size grid (N = 20736) in the benchmark's configuration.  Tolerance:
relative L2 of P(t), J(t) and the occupation <= 1e-4 (the split-FP16 bar of the method).
"""
import numpy as np
import pytest

import workloads as wl
from oracle import channel as oc
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om
from oracle import propagate as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2502_05635_gb300 as tg  # noqa: E402

SPLIT = tg.FLAG_RESET | tg.FLAG_SPLIT_F16
TOL = 1e-4


def _ctx(p):
    return tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)


def _pulses(B, seed):
    """Seeded pulses that peak within the first 60 steps (dt = 0.2)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(B):
        ang = rng.uniform(0.0, np.pi)
        out.append(wl.Pulse(E0=float(10.0 ** rng.uniform(-3.5, -2.2)), omega=float(rng.uniform(0.08, 0.15)),
                            t0=float(rng.uniform(3.0, 8.0)), sigma=float(rng.uniform(1.5, 4.0)),
                            dir_x=float(np.cos(ang)), dir_y=float(np.sin(ang))))
    return out


def _factors(p, rank, ranks_seed=None):
    mdl = om.Model(p)
    P = p.Nb ** 2
    D, U, S, V = oc.channel_svd(ok.dense_kernel(mdl), p.Nb, rank)
    ranks = None
    if ranks_seed is not None:
        ranks = np.random.default_rng(ranks_seed).integers(0, rank + 1, (P, P)).astype(np.int32)
        np.fill_diagonal(ranks, 0)
        mask = np.arange(rank)[None, None, :] < ranks[:, :, None]
        U, V, S = U * mask[:, :, None, :], V * mask[:, :, None, :], S * mask
    return mdl, (D, U, S, V), ranks


def _check_vs_oracle(mdl, fac, got, pulses, steps, dt=0.2):
    D, U, S, V = fac
    apply = lambda v: oc.apply_channel(D, U, S, V, v)  # noqa: E731
    for b, (q, T) in enumerate(zip(pulses, steps)):
        if T == 0:
            assert np.all(np.isnan(got[1:, b]))
            continue
        s = op.half_step_samples(q, dt, T)
        ref, _ = op.rk4(mdl, apply, s, dt, T, direction=(q.dir_x, q.dir_y))
        assert np.abs(ref[:, 0]).max() > 1e-9
        for j in range(3):
            assert op.rel_l2(got[:T + 1, b, j], ref[:, j]) < TOL, (b, j, op.rel_l2(got[:T + 1, b, j], ref[:, j]))
        assert np.all(np.isnan(got[T + 1:, b]))


@pytest.mark.parametrize("L,nc,rank,per_channel", [(12, 1, 9, False), (9, 2, 7, True), (6, 2, 5, False),
                                                   (5, 1, 3, True), (7, 2, 0, False)],
                         ids=["nb2-L12", "nb4-L9-per-channel", "nb4-L6", "nb2-L5-per-channel", "nb4-rank0"])
def test_channel_split_f16_vs_oracle(L, nc, rank, per_channel):
    """Uneven lengths (one of zero steps) against the oracle with the same factors; Nk = 144,
    81, 36, 25 and 49: ragged 16-row chunks and 256-row tiles."""
    p = wl.small_model(L, nc)
    mdl, fac, ranks = _factors(p, rank, ranks_seed=L if per_channel else None)
    c = _ctx(p)
    D, U, S, V = fac
    tg.tdagw_set_channel_factors(c.h, U, S, V, D, ranks=ranks)
    pulses = _pulses(6, 100 + L)
    steps = [60, 17, 60, 0, 41, 3]
    got = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, SPLIT)
    _check_vs_oracle(mdl, fac, got, pulses, steps)


def test_channel_split_f16_agrees_with_fp32_batched_and_replays():
    """150 trajectories (three 64-trajectory groups) of uneven length: the split-FP16 run
    against the FP32 batched channel-wise run of the same factors, and a second identical
    call (cached tuning, CUDA-graph replay) reproduces the first bit for bit."""
    p = wl.small_model(9, 2)
    mdl, fac, _ = _factors(p, 6)
    D, U, S, V = fac
    c = _ctx(p)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    B = 150
    pulses = _pulses(B, 7)
    steps = list(np.random.default_rng(8).integers(1, 50, B))
    a = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, SPLIT)
    b = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, SPLIT)
    np.testing.assert_array_equal(a, b)
    ref = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, tg.FLAG_RESET)
    for j, T in enumerate(steps):
        assert op.rel_l2(a[:T + 1, j, 0], ref[:T + 1, j, 0]) < TOL, j
    _check_vs_oracle(mdl, fac, a[:, ::37], pulses[::37], steps[::37])


@pytest.mark.parametrize("rank", [120, 350])
def test_channel_split_f16_long_v_rows(rank):
    """Two bands, Nk = 400, every off-diagonal channel of rank 120 or 350: V segments of 360
    and 1050 columns (two and five 256-column tiles) and U segments of 760 and 1450 columns."""
    p = wl.small_model(20, 1)
    mdl, fac, _ = _factors(p, rank)
    D, U, S, V = fac
    c = _ctx(p)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    pulses = _pulses(3, 40 + rank)
    steps = [40, 25, 40]
    got = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, SPLIT)
    _check_vs_oracle(mdl, fac, got, pulses, steps)


def test_channel_split_f16_new_factors_refresh_tiles():
    """Installing other channel factors remakes the segment tiles: results follow the new
    factors (rank 2 after rank 6)."""
    p = wl.small_model(6, 2)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    c = _ctx(p)
    pulses = _pulses(2, 3)
    steps = [30, 30]
    for rank in (6, 2):
        fac = oc.channel_svd(K, p.Nb, rank)
        D, U, S, V = fac
        tg.tdagw_set_channel_factors(c.h, U, S, V, D)
        got = c.propagate_batch(pulses, steps, 0.2, tg.CHANNEL, SPLIT)
        _check_vs_oracle(mdl, fac, got, pulses, steps)


def test_full_size_channel_split_f16():
    """N = 20736 (four bands, 36 x 36), the oracle's exact channel factors at rank 65 (5 % of
    Nk), 64 trajectories of early pulses for 30 steps in the benchmark's launch: two sampled
    trajectories against the oracle's propagation with the same factors, all of them
    against the FP32 batched channel-wise run."""
    w = wl.mos2size_channel()
    mdl = om.Model(w.model)
    D, U, S, V = oc.channel_svd_from_model(mdl, w.rank)
    c = _ctx(w.model)
    tg.tdagw_set_channel_factors(c.h, U, S, V, D)
    B, T = 64, 30
    pulses = list(wl.early_pulses(B))
    got = c.propagate_batch(pulses, [T] * B, w.dt, tg.CHANNEL, SPLIT)
    ref32 = c.propagate_batch(pulses, [T] * B, w.dt, tg.CHANNEL, tg.FLAG_RESET)
    for b in range(B):
        assert op.rel_l2(got[:, b, 0], ref32[:, b, 0]) < TOL, b
    apply = lambda v: oc.apply_channel(D, U, S, V, v)  # noqa: E731
    for b in (0, 41):
        q = pulses[b]
        s = op.half_step_samples(q, w.dt, T)
        ref, _ = op.rk4(mdl, apply, s, w.dt, T, direction=(q.dir_x, q.dir_y))
        for j in range(3):
            assert op.rel_l2(got[:, b, j], ref[:, j]) < TOL, (b, j)


@pytest.mark.parametrize("mode", ["lowrank", "channel"])
def test_tensor_core_timeout_is_reported_and_context_survives(mode):
    """Fault injection on the host side of a bounded wait (no GPU fault): the tensor-core
    kernel's grid barrier waits for an arrival that never comes; every wait gives up after
    its 20 ms budget, the copies and MMAs in flight drain, tensor memory is freed, the call
    reports TDAGW_ERR_TIMEOUT at the next synchronisation, and the same context then runs
    the same propagation correctly (against the oracle)."""
    p = wl.small_model(6, 2)
    mdl, fac, _ = _factors(p, 5)
    D, U, S, V = fac
    c = _ctx(p)
    pulses = _pulses(3, 11)
    steps = [20, 12, 20]
    if mode == "channel":
        tg.tdagw_set_channel_factors(c.h, U, S, V, D)
        m, apply = tg.CHANNEL, (lambda v: oc.apply_channel(D, U, S, V, v))  # noqa: E731
    else:
        K = ok.dense_kernel(mdl)
        d, Koff = ok.split_diag_off(K)
        Ul, Sl, Vl = olr.truncated_svd(Koff, 40)
        tg.tdagw_set_factors(c.h, Ul, Sl, Vl, d)
        m = tg.LOWRANK
        apply = lambda v: d * v + Ul @ (Sl * (Vl.conj().T @ v))  # noqa: E731
    tg.tdagw_propagate(c.h, [tg.make_field(q) for q in pulses], steps, 0.2, m,
                       SPLIT | tg.FLAG_TEST_TIMEOUT)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_sync(c.h)
    assert e.value.code == tg.ERR_TIMEOUT
    got = c.propagate_batch(pulses, steps, 0.2, m, SPLIT)
    for b, (q, T) in enumerate(zip(pulses, steps)):
        s = op.half_step_samples(q, 0.2, T)
        ref, _ = op.rk4(mdl, apply, s, 0.2, T, direction=(q.dir_x, q.dir_y))
        assert op.rel_l2(got[:T + 1, b, 0], ref[:, 0]) < TOL, b
