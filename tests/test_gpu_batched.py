"""Batched propagation (many pulses, uneven lengths, one persistent launch) vs the oracle.

Each trajectory is compared with the FP64 oracle run of its own pulse and length (same
factors on both sides); entries after a trajectory's last step must be NaN.  Covers several
trajectory groups (B > 32), ragged groups, both band counts, low-rank and dense modes.
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


def _pulses(B, seed):
    rng = np.random.default_rng(seed)
    return [wl.Pulse(E0=float(10 ** rng.uniform(-3, -2)), omega=float(rng.uniform(0.06, 0.16)),
                     t0=float(rng.uniform(5, 20)), sigma=float(rng.uniform(3, 10)),
                     dir_x=float(np.cos(th)), dir_y=float(np.sin(th)))
            for th in rng.uniform(0, np.pi, B)]


def _check(got, mdl, apply, pulses, steps, dt, tol):
    assert got.shape == (max(steps) + 1, len(steps), 3)
    for b, (p, T) in enumerate(zip(pulses, steps)):
        s = op.half_step_samples(p, dt, T)
        ref, _ = op.rk4(mdl, apply, s, dt, T, direction=(p.dir_x, p.dir_y))
        for j in range(3):
            e = op.rel_l2(got[:T + 1, b, j], ref[:, j])
            assert e < tol, (b, j, e)
        assert np.all(np.isnan(got[T + 1:, b, :]))


@pytest.mark.parametrize("mode", [tg.LOWRANK, tg.FULL])
def test_batched_uneven_vs_oracle(mode):
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 29)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    steps = [37, 150, 90, 150, 3, 121, 64]
    pulses = _pulses(len(steps), 1)
    got = ctx.propagate_batch(pulses, steps, 0.2, mode)
    apply = (lambda v: olr.apply_lowrank(d, U, S, V, v)) if mode == tg.LOWRANK else (lambda v: K @ v)
    _check(got, mdl, apply, pulses, steps, 0.2, 1e-5)


def test_batched_many_groups_seeded_factors():
    """B = 45 (two or more trajectory groups, ragged), N = 2304, rank 256."""
    p = wl.small_model(24, 1)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, 256, seed=4)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    rng = np.random.default_rng(9)
    steps = [int(x) for x in rng.integers(10, 60, 45)]
    pulses = _pulses(45, 2)
    got = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK)
    sel = [0, 7, 19, 30, 44]
    for b in sel:
        T = steps[b]
        s = op.half_step_samples(pulses[b], 0.2, T)
        ref, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, 0.2, T,
                        direction=(pulses[b].dir_x, pulses[b].dir_y))
        assert op.rel_l2(got[:T + 1, b, 0], ref[:, 0]) < 1e-5, b
        assert np.all(np.isnan(got[T + 1:, b]))


def test_batched_four_band_matches_single_trajectory_path():
    p = wl.small_model(9, 2)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 64)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    steps = [80, 33, 80]
    pulses = _pulses(3, 3)
    for mode in (tg.LOWRANK, tg.FULL):
        got = ctx.propagate_batch(pulses, steps, 0.2, mode)
        for b in range(3):
            single = ctx.propagate(pulses[b], steps[b], 0.2, mode)
            assert op.rel_l2(got[:steps[b] + 1, b, 0], single[:, 0]) < 1e-6, (mode, b)


def test_batched_rejects_continue_without_reset():
    p = wl.small_model(4, 1)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_propagate(ctx.h, [tg.make_field(wl.Pulse())] * 2, [5, 5], 0.2, tg.FULL, 0)
    assert e.value.code == tg.ERR_UNSUPPORTED


@pytest.mark.parametrize("flags", [0, tg.FLAG_SPLIT_F16])
def test_graph_replay_matches_direct_launch(flags):
    """Batched launches replayed from the context's cached CUDA graph give the same bits as
    direct launches (TDAGW_FLAG_NO_GRAPH), on first capture and on replay."""
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    U, S, V, d = wl.random_factors(mdl.N, 40, seed=2)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    steps = [30, 12, 25]
    pulses = _pulses(3, 8)
    base = tg.FLAG_RESET | flags
    direct = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, base | tg.FLAG_NO_GRAPH)
    first = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, base)
    again = ctx.propagate_batch(pulses, steps, 0.2, tg.LOWRANK, base)
    np.testing.assert_array_equal(np.nan_to_num(first, nan=7.0), np.nan_to_num(direct, nan=7.0))
    np.testing.assert_array_equal(np.nan_to_num(again, nan=7.0), np.nan_to_num(direct, nan=7.0))


def test_sweep_full_size_sampled_vs_oracle():
    """The field-sweep workload at full size in the benchmark's launch configuration (N =
    2304, rank 256, 256 trajectories of 500-4000 steps, one launch), FP32 and split-FP16,
    seeded factors on both sides: the three shortest trajectories over their whole length
    against the FP64 oracle, and the NaN padding after every trajectory's end."""
    w = wl.sweep_nb2_l24()
    mdl = om.Model(w.model)
    U, S, V, d = wl.random_factors(mdl.N, w.rank, seed=23)
    ctx = tg.Context(w.model, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    fp32 = ctx.propagate_batch(w.pulses, w.steps, w.dt, tg.LOWRANK)
    split = ctx.propagate_batch(w.pulses, w.steps, w.dt, tg.LOWRANK, tg.FLAG_RESET | tg.FLAG_SPLIT_F16)
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
    for b in np.argsort(w.steps)[:3]:
        T, q = int(w.steps[b]), w.pulses[b]
        s = op.half_step_samples(q, w.dt, T)
        ref, _ = op.rk4(mdl, apply, s, w.dt, T, direction=(q.dir_x, q.dir_y))
        assert op.rel_l2(fp32[:T + 1, b, 0], ref[:, 0]) < 1e-5, b
        assert op.rel_l2(split[:T + 1, b, 0], ref[:, 0]) < 1e-4, b
    for b, T in enumerate(w.steps):
        assert np.all(np.isnan(fp32[T + 1:, b])) and np.all(np.isnan(split[T + 1:, b]))


@pytest.mark.parametrize("mode,flags", [(tg.LOWRANK, tg.FLAG_RESET), (tg.FULL, tg.FLAG_RESET),
                                        (tg.LOWRANK, tg.FLAG_RESET | tg.FLAG_SPLIT_F16)])
def test_zero_step_trajectories_inside_a_batch(mode, flags):
    """Trajectories of zero steps next to running ones: their only row is the equilibrium
    observables at t = 0 and every later row is NaN; the others match the oracle."""
    p = wl.small_model(12, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 29)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    steps = [40, 0, 25, 0, 7]
    pulses = _pulses(len(steps), 5)
    got = ctx.propagate_batch(pulses, steps, 0.2, mode, flags)
    assert got.shape == (41, 5, 3)
    eq = op.observables(mdl, np.zeros(mdl.N, complex))
    apply = (lambda v: olr.apply_lowrank(d, U, S, V, v)) if mode == tg.LOWRANK else (lambda v: K @ v)
    tol = 1e-4 if flags & tg.FLAG_SPLIT_F16 else 1e-5
    for b, (pl, T) in enumerate(zip(pulses, steps)):
        if T == 0:
            np.testing.assert_allclose(got[0, b], eq, atol=1e-7)
            assert np.all(np.isnan(got[1:, b]))
            continue
        s = op.half_step_samples(pl, 0.2, T)
        ref, _ = op.rk4(mdl, apply, s, 0.2, T, direction=(pl.dir_x, pl.dir_y))
        assert op.rel_l2(got[:T + 1, b, 0], ref[:, 0]) < tol, b
        assert np.all(np.isnan(got[T + 1:, b]))
    ctx.close()


@pytest.mark.parametrize("mode", [tg.LOWRANK, tg.FULL])
def test_batched_timeout_is_reported_and_context_survives(mode):
    """Fault injection on the host side of a bounded wait (no GPU fault): the FP32 batched
    kernel's grid barrier waits for an arrival that never comes; the call reports
    TDAGW_ERR_TIMEOUT at the next synchronisation and the same context then runs the same
    batch correctly (against the oracle)."""
    p = wl.small_model(6, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 20)
    c = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(c.h, U, S, V, d)
    pulses = _pulses(5, 21)
    steps = [30, 9, 30, 17, 1]
    tg.tdagw_propagate(c.h, [tg.make_field(q) for q in pulses], steps, 0.2, mode,
                       tg.FLAG_RESET | tg.FLAG_TEST_TIMEOUT)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_sync(c.h)
    assert e.value.code == tg.ERR_TIMEOUT
    got = c.propagate_batch(pulses, steps, 0.2, mode)
    if mode == tg.FULL:
        apply = lambda v: K @ v  # noqa: E731
    else:
        apply = lambda v: d * v + U @ (S * (V.conj().T @ v))  # noqa: E731
    _check(got, mdl, apply, pulses, steps, 0.2, 1e-5)
