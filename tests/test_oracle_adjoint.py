"""Pins of the oracle's discrete adjoint: vector-Jacobian identity, objective derivative,
and central finite differences of the FP64 forward (field samples and pulse parameters).
No GPU."""
import numpy as np
import pytest

import workloads as wl
from oracle import adjoint as oa
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om
from oracle import propagate as op


@pytest.fixture(scope="module")
def setup():
    p = wl.small_model(4, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    return mdl, K


def _inner(a, b):
    return float(np.real(np.vdot(a, b)))


def test_vjp_dot_product_identity(setup):
    mdl, K = setup
    rng = np.random.default_rng(0)
    X = wl.random_state(mdl.N, 1, 0.05)
    g = wl.random_state(mdl.N, 2, 1.0)
    dX = wl.random_state(mdl.N, 3, 1.0)
    E, direction = 0.003, (0.6, 0.8)
    f = lambda x, e: op.rhs(mdl, lambda v: K @ v, e * direction[0], e * direction[1], x)
    eps = 1e-6
    jdx = (f(X + eps * dX, E) - f(X - eps * dX, E)) / (2 * eps)
    jde = (f(X, E + eps) - f(X, E - eps)) / (2 * eps)
    xbar, ebar = oa.vjp(mdl, lambda v: K @ v, lambda v: K.conj().T @ v, E, direction, X, g)
    assert abs(_inner(g, jdx) - _inner(xbar, dX)) < 1e-8 * abs(_inner(g, jdx))
    assert abs(_inner(g, jde) - ebar) < 1e-8 * abs(ebar)


def test_objective_derivative():
    rng = np.random.default_rng(4)
    P = rng.standard_normal(101)
    J, dJ = oa.spectral_objective(P, 0.2, 0.1)
    for n in (0, 17, 100):
        e = np.zeros_like(P)
        e[n] = 1e-6
        fd = (oa.spectral_objective(P + e, 0.2, 0.1)[0] - oa.spectral_objective(P - e, 0.2, 0.1)[0]) / 2e-6
        assert abs(fd - dJ[n]) < 1e-7 * max(1.0, abs(fd))


def _J_of_samples(mdl, apply, samples, dt, T, direction, w0):
    obs, _ = op.rk4(mdl, apply, samples, dt, T, direction=direction)
    return oa.spectral_objective(obs[:, 0], dt, w0)[0]


@pytest.mark.parametrize("lowrank", [False, True])
def test_adjoint_field_samples_vs_finite_differences(setup, lowrank):
    mdl, K = setup
    if lowrank:
        d, Koff = ok.split_diag_off(K)
        U, S, V = olr.truncated_svd(Koff, 9)
        apply = lambda v: olr.apply_lowrank(d, U, S, V, v)
        applyH = lambda v: np.conj(d) * v + V @ (S * (U.conj().T @ v))
    else:
        apply, applyH = (lambda v: K @ v), (lambda v: K.conj().T @ v)
    pulse = wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0, dir_x=0.8, dir_y=0.6)
    dt, T = 0.2, 60
    direction = (pulse.dir_x, pulse.dir_y)
    samples = op.half_step_samples(pulse, dt, T)
    obs, _ = op.rk4(mdl, apply, samples, dt, T, direction=direction)
    _, dJdP = oa.spectral_objective(obs[:, 0], dt, pulse.omega)
    gE = oa.adjoint(mdl, apply, applyH, samples, dt, T, direction, dJdP)
    for j in (0, 1, 31, 60, 61, 119, 120):
        hj = 1e-6 * max(1e-3, abs(samples[j]))
        sp, sm = samples.copy(), samples.copy()
        sp[j] += hj
        sm[j] -= hj
        fd = (_J_of_samples(mdl, apply, sp, dt, T, direction, pulse.omega)
              - _J_of_samples(mdl, apply, sm, dt, T, direction, pulse.omega)) / (2 * hj)
        assert abs(fd - gE[j]) <= 1e-5 * np.abs(gE).max(), (j, fd, gE[j])


def test_adjoint_pulse_parameters_vs_finite_differences(setup):
    mdl, K = setup
    apply, applyH = (lambda v: K @ v), (lambda v: K.conj().T @ v)
    pulse = wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0)
    dt, T = 0.2, 60
    J, gp, _ = oa.objective_and_gradients(mdl, apply, applyH, pulse, dt, T)
    import dataclasses
    for i, name in enumerate(("E0", "omega", "t0", "sigma")):
        v = getattr(pulse, name)
        h = 1e-6 * abs(v)
        Jp = _J_of_samples(mdl, apply, op.half_step_samples(dataclasses.replace(pulse, **{name: v + h}), dt, T),
                           dt, T, (1.0, 0.0), pulse.omega)
        Jm = _J_of_samples(mdl, apply, op.half_step_samples(dataclasses.replace(pulse, **{name: v - h}), dt, T),
                           dt, T, (1.0, 0.0), pulse.omega)
        fd = (Jp - Jm) / (2 * h)
        assert abs(fd - gp[i]) <= 1e-5 * abs(gp[i]) + 1e-12 * abs(J), (name, fd, gp[i])


def test_adjoint_all_observables_vs_finite_differences(setup):
    """Objective weighting P, J and the c1 occupation: the direct terms of J and occ."""
    mdl, K = setup
    apply, applyH = (lambda v: K @ v), (lambda v: K.conj().T @ v)
    pulse = wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0, dir_x=0.6, dir_y=0.8)
    dt, T = 0.2, 40
    direction = (pulse.dir_x, pulse.dir_y)
    samples = op.half_step_samples(pulse, dt, T)
    rng = np.random.default_rng(11)
    W = rng.standard_normal((T + 1, 3))
    W[:, 2] *= 50.0                                     # occupations are small; weight them up

    def J_of(s):
        obs, _ = op.rk4(mdl, apply, s, dt, T, direction=direction)
        return float(np.sum(W * obs ** 2))

    obs, _ = op.rk4(mdl, apply, samples, dt, T, direction=direction)
    G = 2 * W * obs
    gE = oa.adjoint(mdl, apply, applyH, samples, dt, T, direction, G[:, 0], G[:, 1], G[:, 2])
    for j in (0, 7, 40, 41, 79, 80):
        hj = 1e-6 * max(1e-3, abs(samples[j]))
        sp, sm = samples.copy(), samples.copy()
        sp[j] += hj
        sm[j] -= hj
        fd = (J_of(sp) - J_of(sm)) / (2 * hj)
        assert abs(fd - gE[j]) <= 1e-5 * np.abs(gE).max(), (j, fd, gE[j])
    # each observable's direct term matters: dropping one changes the gradient
    for z in range(3):
        Gz = G.copy()
        Gz[:, z] = 0
        gz = oa.adjoint(mdl, apply, applyH, samples, dt, T, direction, Gz[:, 0], Gz[:, 1], Gz[:, 2])
        assert np.abs(gz - gE).max() > 1e-3 * np.abs(gE).max()


def test_observable_gradients_match_observables(setup):
    """<grad O, X> reproduces the observable's linear part for a random state."""
    mdl, _ = setup
    X = wl.random_state(mdl.N, 5, 0.1)
    base = op.observables(mdl, np.zeros(mdl.N, dtype=np.complex128))
    got = op.observables(mdl, X) - base
    for g, v in zip(oa.observable_gradients(mdl), got):
        assert abs(_inner(g, X) - v) < 1e-13


@pytest.mark.parametrize("lowrank", [False, True])
def test_adjoint_matches_reverse_mode_ad_of_the_forward(setup, lowrank):
    """The hand-derived discrete adjoint against torch float64 reverse-mode AD of the RK4
    forward written from the equation of motion (no finite-difference noise: agreement to
    rounding).  The torch forward is first checked against the oracle's P(t)."""
    torch = pytest.importorskip("torch")
    mdl, K = setup
    if lowrank:
        d, Koff = ok.split_diag_off(K)
        U, S, V = olr.truncated_svd(Koff, 9)
        Kt = np.diag(d) + (U * S) @ V.conj().T
    else:
        Kt = K
    apply, applyH = (lambda v: Kt @ v), (lambda v: Kt.conj().T @ v)
    pulse = wl.Pulse(E0=0.02, omega=0.15, t0=6.0, sigma=3.0, dir_x=0.8, dir_y=0.6)
    dt, T = 0.2, 50
    direction = (pulse.dir_x, pulse.dir_y)
    samples = op.half_step_samples(pulse, dt, T)
    obs, _ = op.rk4(mdl, apply, samples, dt, T, direction=direction)
    _, dJdP = oa.spectral_objective(obs[:, 0], dt, pulse.omega)
    gE = oa.adjoint(mdl, apply, applyH, samples, dt, T, direction, dJdP)

    Nk, Nb = mdl.Nk, mdl.Nb
    c = lambda a: torch.as_tensor(np.array(a), dtype=torch.complex128)  # noqa: E731
    Kq = c(Kt)
    Dq = c(direction[0] * mdl.dx + direction[1] * mdl.dy)
    H0 = torch.diag_embed(c(mdl.eps))
    R0 = torch.diag_embed(c(np.broadcast_to(mdl.occ, (Nk, Nb))))
    dxT = c(np.swapaxes(mdl.dx, 1, 2))
    s = torch.tensor(samples, dtype=torch.float64, requires_grad=True)

    def f(X, E):                                   # -i [H0 + E D + (K X), rho0 + X] per k
        H = H0 + E * Dq + (Kq @ X.reshape(-1)).reshape(Nk, Nb, Nb)
        rho = R0 + X
        return -1j * (H @ rho - rho @ H)

    def pol(X):                                    # P_x = (1/Nk) Re sum_k Tr(rho_k d_k)
        return ((R0 + X) * dxT).sum().real / Nk

    X = torch.zeros((Nk, Nb, Nb), dtype=torch.complex128)
    P = [pol(X)]
    for n in range(T):
        k1 = f(X, s[2 * n])
        k2 = f(X + 0.5 * dt * k1, s[2 * n + 1])
        k3 = f(X + 0.5 * dt * k2, s[2 * n + 1])
        k4 = f(X + dt * k3, s[2 * n + 2])
        X = X + (dt / 6.0) * (k1 + 2 * k2 + 2 * k3 + k4)
        P.append(pol(X))
    P = torch.stack(P)
    np.testing.assert_allclose(P.detach().numpy(), obs[:, 0], rtol=0, atol=1e-14 * np.abs(obs[:, 0]).max())
    # the spectral objective on the DFT grid of the T + 1 samples (weights fixed)
    w = 2 * np.pi * np.arange(T + 1) / ((T + 1) * dt)
    Em = torch.as_tensor(np.exp(-1j * np.outer(w, np.arange(T + 1) * dt)) * dt)
    wgt = torch.as_tensor(oa.harmonic_window(w, pulse.omega))
    F = Em @ P.to(torch.complex128)
    J = (wgt * F.abs() ** 2).sum()
    J.backward()
    g_ad = s.grad.numpy()
    assert np.abs(gE).max() > 0
    np.testing.assert_allclose(gE, g_ad, rtol=0, atol=1e-10 * np.abs(g_ad).max())
