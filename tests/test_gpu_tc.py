"""Split-FP16 tensor-core batched propagation (TDAGW_FLAG_SPLIT_F16) vs the FP64 oracle and
vs the FP32 batched path, with the same factors on every side.

The split-FP16 products carry about 22 significant bits (FP32 accumulation), so P(t) must
match the oracle to the split-FP16 bound 1e-4 (relative L2 over the run) and in practice
sits at the FP32 level.  Cases: ragged row tiles (N not a multiple of 256), several
trajectory groups (B > 64), ranks spanning one to three 256-row tiles of V^H, both band
counts, field strengths over two decades in one batch, lengths ending at different steps,
the tuned work split of the launch.
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

SPLIT = tg.FLAG_RESET | tg.FLAG_SPLIT_F16


def _pulses(B, seed, lo=-4.0, hi=-2.0):
    rng = np.random.default_rng(seed)
    return [wl.Pulse(E0=float(10 ** rng.uniform(lo, hi)), omega=float(rng.uniform(0.06, 0.16)),
                     t0=float(rng.uniform(5, 20)), sigma=float(rng.uniform(3, 10)),
                     dir_x=float(np.cos(th)), dir_y=float(np.sin(th)))
            for th in rng.uniform(0, np.pi, B)]


def _oracle(mdl, apply, pulse, T, dt=0.2):
    s = op.half_step_samples(pulse, dt, T)
    ref, _ = op.rk4(mdl, apply, s, dt, T, direction=(pulse.dir_x, pulse.dir_y))
    return ref


def _ctx(p, U, S, V, d):
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    return ctx


@pytest.mark.parametrize("L,nc,rank", [(4, 1, 9), (12, 1, 29), (6, 2, 200)])
def test_split_f16_vs_oracle(L, nc, rank):
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, rank)
    ctx = _ctx(p, U, S, V, d)
    steps = [120, 37, 120, 80, 5]
    pulses = _pulses(len(steps), 3)
    got = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
    for b, (q, T) in enumerate(zip(pulses, steps)):
        ref = _oracle(mdl, apply, q, T)
        for j in range(3):
            e = op.rel_l2(got[:T + 1, b, j], ref[:, j])
            assert e < 1e-4, (b, j, e)
        assert np.all(np.isnan(got[T + 1:, b]))


def test_split_f16_single_trajectory():
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, 64, seed=5)
    ctx = _ctx(p, U, S, V, d)
    q = wl.Pulse(E0=0.01, omega=0.12, t0=10.0, sigma=5.0)
    got = ctx.propagate_batch([q], [150], 0.2, tg.LOWRANK, SPLIT)
    ref = _oracle(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), q, 150)
    assert op.rel_l2(got[:, 0], ref[:, 0]) < 1e-4


@pytest.mark.parametrize("rank", [64, 520])
def test_split_f16_many_groups_vs_fp32(rank):
    """B = 150 (three trajectory groups), field strengths 1e-4..1e-2; rank 520 uses three
    256-row tiles of V^H."""
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, rank, seed=6)
    ctx = _ctx(p, U, S, V, d)
    rng = np.random.default_rng(10)
    steps = [int(x) for x in rng.integers(5, 40, 150)]
    pulses = _pulses(150, 4)
    got = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    fp32 = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK)
    for b, T in enumerate(steps):
        e = op.rel_l2(got[:T + 1, b, 0], fp32[:T + 1, b, 0])
        assert e < 1e-4, (b, e)
        assert np.all(np.isnan(got[T + 1:, b]))
    for b in (0, 77, 149):
        ref = _oracle(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), pulses[b], steps[b])
        assert op.rel_l2(got[:steps[b] + 1, b, 0], ref[:, 0]) < 1e-4, b


def test_split_f16_after_compress_precision1():
    p = wl.small_model(12, 1)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_compress_svd(ctx.h, 48, 32, 2, 1, precision=1)
    pulses = _pulses(6, 5)
    steps = [60, 50, 40, 30, 20, 10]
    got = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    fp32 = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK)
    for b, T in enumerate(steps):
        assert op.rel_l2(got[:T + 1, b, 0], fp32[:T + 1, b, 0]) < 1e-4, b


def test_split_f16_refreshes_after_new_factors():
    """The tiled copy follows tdagw_set_factors."""
    p = wl.small_model(4, 1)
    mdl = om.Model(p)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    q = wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0)
    for seed in (7, 8):
        U, S, V, d = wl.random_factors(mdl.N, 12, seed=seed)
        tg.tdagw_set_factors(ctx.h, U, S, V, d)
        got = ctx.propagate_batch([q, q], [40, 40], 0.2, tg.LOWRANK, SPLIT)
        ref = _oracle(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), q, 40)
        assert op.rel_l2(got[:, 1, 0], ref[:, 0]) < 1e-4


def test_split_f16_errors():
    p = wl.small_model(4, 1)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, 8, seed=1)
    ctx = _ctx(p, U, S, V, d)
    q = wl.Pulse()
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(ctx.h, [tg.make_field(q)], [5], 0.2, tg.FULL, SPLIT)
    assert e.value.code == tg.ERR_INVALID_ARG
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(ctx.h, [tg.make_field(q)], [5], 0.2, tg.LOWRANK, tg.FLAG_SPLIT_F16)
    assert e.value.code == tg.ERR_UNSUPPORTED
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_compress_svd(ctx.h, 8, 8, 1, 1, precision=2)
    assert e.value.code == tg.ERR_INVALID_ARG
    c128 = tg.Context(p, tg.C128, stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_compress_svd(c128.h, 8, 8, 1, 1, precision=1)
    assert e.value.code == tg.ERR_UNSUPPORTED


def test_split_f16_tuned_work_split_vs_oracle_and_replay():
    """The work split of the tensor-core launch (trajectory groups of the U product,
    K-ranges of the V^H X product) is tuned by timing on the first long enough call and
    cached: the tuned call matches the oracle, and a second call (cached split, replayed
    graph) reproduces it bitwise."""
    p = wl.small_model(12, 2)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, 96, seed=9)
    ctx = _ctx(p, U, S, V, d)
    pulses = _pulses(20, 6)
    steps = [int(x) for x in np.random.default_rng(3).integers(10, 30, 20)]
    one = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    two = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    assert np.array_equal(one, two, equal_nan=True)
    ref = _oracle(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), pulses[0], steps[0])
    assert op.rel_l2(one[:steps[0] + 1, 0, 0], ref[:, 0]) < 1e-4


def test_precision_study_size_vs_oracle():
    """The precision-study size (four-band 48 x 48, N = 36864, rank 2048, B = 64): split-FP16
    and FP32 batched runs of 64 early pulses (uneven lengths) against the FP64 oracle on two
    trajectories, with the same seeded factors on every side."""
    w = wl.prec_nb4_l48()
    mdl = om.Model(w.model)
    U, S, V, d = wl.random_factors(mdl.N, w.rank, seed=3)
    ctx = _ctx(w.model, U, S, V, d)
    rng = np.random.default_rng(21)
    pulses = [wl.Pulse(E0=float(10 ** rng.uniform(-4, -2)), omega=float(rng.uniform(0.06, 0.16)),
                       t0=float(rng.uniform(0.5, 1.0)), sigma=float(rng.uniform(0.4, 0.8)),
                       dir_x=float(np.cos(th)), dir_y=float(np.sin(th)))
              for th in rng.uniform(0, np.pi, 64)]
    steps = [6] * 32 + [4] * 32
    split = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, SPLIT)
    fp32 = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK)
    for b, T in enumerate(steps):
        assert op.rel_l2(split[:T + 1, b, 0], fp32[:T + 1, b, 0]) < 1e-4, b
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
    for b in (0, 63):
        ref = _oracle(mdl, apply, pulses[b], steps[b])
        assert op.rel_l2(fp32[:steps[b] + 1, b, 0], ref[:, 0]) < 1e-5, b
        assert op.rel_l2(split[:steps[b] + 1, b, 0], ref[:, 0]) < 1e-4, b


def test_precision_study_rsvd_factors_200_steps_vs_oracle():
    """The precision study as configured: four-band 48 x 48 model (N = 36864), rank 2048
    from the GPU's randomised SVD of K^off (oversampling 64, two power iterations, FP64
    orthogonalisation) emitted as split-FP16 tiles, 64 trajectories from the sweep
    distributions, 200 RK4 steps.  Split-FP16 with Kahan-compensated RK4, FP32 with and
    without compensation, each against the FP64 oracle run with the same factors
    (tdagw_get_factors) on the two trajectories whose pulses are widest (largest field in
    the prefix), and split-FP16 against FP32 on all 64."""
    w = wl.prec_nb4_l48()
    mdl = om.Model(w.model)
    c = tg.Context(w.model, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_compress_svd(c.h, w.rank, w.oversample, w.power_iters, wl.SKETCH_SEED, precision=1)
    U, S, V, d = tg.tdagw_get_factors(c.h)
    T, B = 200, w.B
    steps = [T] * B
    split = c.propagate_batch(w.pulses, steps, w.dt, tg.LOWRANK, SPLIT)
    fp32 = c.propagate_batch(w.pulses, steps, w.dt, tg.LOWRANK, tg.FLAG_RESET)
    plain = c.propagate_batch(w.pulses, steps, w.dt, tg.LOWRANK, tg.FLAG_RESET | tg.FLAG_NO_KAHAN)
    for b in range(B):
        assert op.rel_l2(split[:, b, 0], fp32[:, b, 0]) < 1e-4, b
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)  # noqa: E731
    widest = np.argsort([p.sigma for p in w.pulses])[-2:]
    for b in widest:
        ref = _oracle(mdl, apply, w.pulses[b], T, w.dt)
        assert np.abs(ref[:, 0]).max() > 0
        e_split = op.rel_l2(split[:, b, 0], ref[:, 0])
        e_fp32 = op.rel_l2(fp32[:, b, 0], ref[:, 0])
        e_plain = op.rel_l2(plain[:, b, 0], ref[:, 0])
        print(f"trajectory {b}: split-FP16 {e_split:.2e}, FP32 {e_fp32:.2e}, FP32 uncompensated {e_plain:.2e}")
        assert e_split < 1e-4 and e_fp32 < 1e-5 and e_plain < 1e-5, (b, e_split, e_fp32, e_plain)
    c.close()
