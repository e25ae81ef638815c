"""GPU discrete adjoint (checkpointed batched RK4) vs the FP64 oracle adjoint.

Both adjoints take the same objective derivative (the oracle's spectral objective of the
oracle's P(t)); the GPU field-sample and pulse-parameter gradients must match the oracle's
to 1e-4 (relative L2 / max), through several checkpoint segments and uneven lengths.
"""
import dataclasses

import numpy as np
import pytest

import workloads as wl
from oracle import adjoint as oa
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om
from oracle import propagate as op

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2502_05635_gb300 as tg  # noqa: E402


def _case(L, nc, rank):
    p = wl.small_model(L, nc)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, rank)
    return p, mdl, K, d, U, S, V


PULSES = [wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0),
          wl.Pulse(E0=0.015, omega=0.11, t0=4.0, sigma=2.5, dir_x=0.6, dir_y=0.8),
          wl.Pulse(E0=0.01, omega=0.13, t0=5.0, sigma=4.0)]


@pytest.mark.parametrize("mode,split", [(tg.LOWRANK, False), (tg.FULL, False), (tg.LOWRANK, True)],
                         ids=["lowrank", "full", "lowrank-split-f16"])
@pytest.mark.parametrize("L,nc,rank", [(4, 1, 9), (3, 2, 20)])
def test_adjoint_matches_oracle(mode, split, L, nc, rank):
    """split: the checkpointed forward and the segment recomputes on the tensor cores
    (split-FP16 factors), the reverse stages with the FP32 factors."""
    p, mdl, K, d, U, S, V = _case(L, nc, rank)
    if mode == tg.LOWRANK:
        apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
        applyH = lambda v: np.conj(d) * v + V @ (S * (U.conj().T @ v))
    else:
        apply, applyH = (lambda v: K @ v), (lambda v: K.conj().T @ v)
    dt, steps = 0.2, [60, 45, 60]
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    tg.tdagw_propagate(ctx.h, [tg.make_field(q) for q in PULSES], steps, dt, mode,
                       tg.FLAG_RESET | tg.FLAG_CHECKPOINT | (tg.FLAG_SPLIT_F16 if split else 0))
    got_obs = tg.tdagw_observables(ctx.h, B=3)
    dJ = np.zeros((61, 3, 3))
    refs = []
    for b, (q, T) in enumerate(zip(PULSES, steps)):
        s = op.half_step_samples(q, dt, T)
        obs, _ = op.rk4(mdl, apply, s, dt, T, direction=(q.dir_x, q.dir_y))
        assert op.rel_l2(got_obs[:T + 1, b, 0], obs[:, 0]) < (1e-4 if split else 1e-5)
        _, dJdP = oa.spectral_objective(obs[:, 0], dt, q.omega)
        dJ[:T + 1, b, 0] = dJdP
        gE = oa.adjoint(mdl, apply, applyH, s, dt, T, (q.dir_x, q.dir_y), dJdP)
        gp = oa.pulse_param_jacobian(q, dt, T).T @ gE
        refs.append((gE, gp))
    gE_gpu, gp_gpu = tg.tdagw_adjoint(ctx.h, dJ, 60, 3)
    for b, (T, (gE, gp)) in enumerate(zip(steps, refs)):
        e = np.linalg.norm(gE_gpu[:2 * T + 1, b] - gE) / np.linalg.norm(gE)
        assert e < 1e-4, (b, e)
        assert np.all(gE_gpu[2 * T + 1:, b] == 0)
        np.testing.assert_allclose(gp_gpu[b], gp, rtol=1e-4, atol=1e-4 * np.abs(gp).max())


def test_autograd_function_gradient():
    p, mdl, K, d, U, S, V = _case(4, 1, 9)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    dt, steps = 0.2, [50, 50]
    params = torch.tensor([[q.E0, q.omega, q.t0, q.sigma] for q in PULSES[:2]],
                          dtype=torch.float64, requires_grad=True)
    P = tg.propagate_autograd(ctx, params, PULSES[:2], steps, dt, tg.LOWRANK)
    w = torch.linspace(0.5, 1.5, P.shape[0], dtype=torch.float64)[:, None]
    loss = (w * P ** 2).sum()
    loss.backward()
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
    applyH = lambda v: np.conj(d) * v + V @ (S * (U.conj().T @ v))
    for b in range(2):
        q = PULSES[b]
        s = op.half_step_samples(q, dt, 50)
        obs, _ = op.rk4(mdl, apply, s, dt, 50, direction=(q.dir_x, q.dir_y))
        dJdP = 2 * w[:, 0].numpy() * obs[:, 0]
        gE = oa.adjoint(mdl, apply, applyH, s, dt, 50, (q.dir_x, q.dir_y), dJdP)
        gp = oa.pulse_param_jacobian(q, dt, 50).T @ gE
        np.testing.assert_allclose(params.grad[b].numpy(), gp, rtol=1e-4, atol=1e-4 * np.abs(gp).max())


def test_adjoint_requires_checkpointed_run():
    p = wl.small_model(4, 1)
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    ctx.propagate(wl.Pulse(), 10, 0.2, tg.FULL)
    with pytest.raises(tg.TdagwError) as e:
        tg.tdagw_adjoint(ctx.h, np.zeros((11, 1, 3)), 10, 1)
    assert e.value.code == tg.ERR_INVALID_ARG


@pytest.mark.parametrize("mode", [tg.LOWRANK, tg.FULL])
def test_adjoint_all_observables(mode):
    """Objective sum_n,z W_nz obs_nz^2 over P, J and occ: exercises every direct term."""
    p, mdl, K, d, U, S, V = _case(4, 1, 9)
    if mode == tg.LOWRANK:
        apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
        applyH = lambda v: np.conj(d) * v + V @ (S * (U.conj().T @ v))
    else:
        apply, applyH = (lambda v: K @ v), (lambda v: K.conj().T @ v)
    dt, steps = 0.2, [40, 33]
    ctx = tg.Context(p, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    tg.tdagw_propagate(ctx.h, [tg.make_field(q) for q in PULSES[1:3]], steps, dt, mode,
                       tg.FLAG_RESET | tg.FLAG_CHECKPOINT)
    rng = np.random.default_rng(12)
    dJ = np.zeros((41, 2, 3))
    refs = []
    for b, (q, T) in enumerate(zip(PULSES[1:3], steps)):
        s = op.half_step_samples(q, dt, T)
        obs, _ = op.rk4(mdl, apply, s, dt, T, direction=(q.dir_x, q.dir_y))
        W = rng.standard_normal((T + 1, 3)) * np.array([1.0, 1.0, 50.0])
        G = 2 * W * obs
        dJ[:T + 1, b] = G
        refs.append(oa.adjoint(mdl, apply, applyH, s, dt, T, (q.dir_x, q.dir_y), G[:, 0], G[:, 1], G[:, 2]))
    gE_gpu, _ = tg.tdagw_adjoint(ctx.h, dJ, 40, 2)
    for b, (T, gE) in enumerate(zip(steps, refs)):
        e = np.linalg.norm(gE_gpu[:2 * T + 1, b] - gE) / np.linalg.norm(gE)
        assert e < 1e-4, (b, e)


@pytest.mark.parametrize("split", [False, True], ids=["fp32", "split-f16"])
def test_adjoint_full_size_vs_oracle(split):
    """The differentiation workload's size (two-band 36 x 36, N = 5184, rank 512, B = 32) with
    pulses that act inside a 60-step window: field-sample and pulse-parameter gradients of
    two trajectories against the FP64 oracle adjoint (seeded factors on both sides); split:
    the checkpointed forward and its recomputes on the tensor cores."""
    w = wl.adj_nb2_l36()
    mdl = om.Model(w.model)
    U, S, V, d = wl.random_factors(mdl.N, w.rank, seed=29)
    ctx = tg.Context(w.model, tg.C64, stream=torch.cuda.current_stream().cuda_stream)
    tg.tdagw_set_factors(ctx.h, U, S, V, d)
    rng = np.random.default_rng(31)
    pulses = [wl.Pulse(E0=float(10 ** rng.uniform(-3.5, -2.5)), omega=float(rng.uniform(0.06, 0.16)),
                       t0=float(rng.uniform(4, 8)), sigma=float(rng.uniform(2, 3)))
              for _ in range(w.B)]
    T, dt = 60, w.dt
    tg.tdagw_propagate(ctx.h, [tg.make_field(q) for q in pulses], [T] * w.B, dt, tg.LOWRANK,
                       tg.FLAG_RESET | tg.FLAG_CHECKPOINT | (tg.FLAG_SPLIT_F16 if split else 0))
    apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
    applyH = lambda v: np.conj(d) * v + V @ (S * (U.conj().T @ v))
    dJ = np.zeros((T + 1, w.B, 3))
    refs = {}
    for b in (0, w.B - 1):
        q = pulses[b]
        s = op.half_step_samples(q, dt, T)
        obs, _ = op.rk4(mdl, apply, s, dt, T)
        _, dJdP = oa.spectral_objective(obs[:, 0], dt, q.omega)
        dJ[:, b, 0] = dJdP
        gE = oa.adjoint(mdl, apply, applyH, s, dt, T, (1.0, 0.0), dJdP)
        refs[b] = (gE, oa.pulse_param_jacobian(q, dt, T).T @ gE)
    gE_gpu, gp_gpu = tg.tdagw_adjoint(ctx.h, dJ, T, w.B)
    for b, (gE, gp) in refs.items():
        assert op.rel_l2(gE_gpu[:, b], gE) < 1e-4, b
        np.testing.assert_allclose(gp_gpu[b], gp, rtol=1e-4, atol=1e-4 * np.abs(gp).max())
