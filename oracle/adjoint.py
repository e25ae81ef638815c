"""Spectral objective of P(t) and its exact discrete adjoint through RK4 (FP64).

Test infrastructure only (see the package header).

Objective (the harmonic-generation analysis of Sec. "SVD acceleration": spectra are
Fourier transforms of P(t) / J(t)).  Readings (the paper gives no objective): for a run of
T steps with samples P_n = P_x(n dt), n = 0..T,
    F(w_j) = sum_n P_n exp(-i w_j n dt) dt,   w_j = 2 pi j / ((T + 1) dt), j = 0..T,
    J = sum_j wgt(w_j) |F(w_j)|^2,   wgt(w) = sum_{h=3..7} exp(-(w - h w0)^2 / (2 (w0/8)^2)),
with w0 the pulse's nominal frequency held fixed (no derivative through the window).

Adjoint: the gradient of J is propagated backwards through the discrete RK4 map exactly
(the adjoint of the scheme, not of the ODE), so it matches finite differences of the
discrete forward to rounding.  With the real inner product <a, b> = Re sum conj(a_i) b_i,
the vector-Jacobian product of f(X) = -i [A(X), rho(X)], A = diag(eps) + E D + K X,
rho = rho0 + X, for a cotangent g is (per k block)
    Xbar = i (A^+ g - g A^+) + K^H [ i (g rho^+ - rho^+ g) ],
    Ebar = <g, -i [D, rho]>.
For a step x' = x + h/6 (k1 + 2 k2 + 2 k3 + k4) with stage inputs X1 = x, X2 = x + h/2 k1,
X3 = x + h/2 k2, X4 = x + h k3 and lam = dJ/dx':
    gk4 = h/6 lam;               mu4 = VJP(X4, gk4)
    gk3 = h/3 lam + h mu4;       mu3 = VJP(X3, gk3)
    gk2 = h/3 lam + h/2 mu3;     mu2 = VJP(X2, gk2)
    gk1 = h/6 lam + h/2 mu2;     mu1 = VJP(X1, gk1)
    dJ/dx = lam + mu1 + mu2 + mu3 + mu4 (+ the direct terms of the observables at step n)
and dJ/dE at the stage samples is the Ebar of each stage (the two middle stages share
the sample at t_n + dt/2).
"""
from __future__ import annotations

import numpy as np

from . import propagate as op


def harmonic_window(w: np.ndarray, w0: float) -> np.ndarray:
    """Weight of the objective around harmonics 3-7 of w0 (a reading: the paper differentiates
    nothing; its spectra, Sec. "SVD acceleration of TD-aGW", are transforms of P(t), J(t))."""
    s = w0 / 8.0
    return sum(np.exp(-((w - h * w0) ** 2) / (2 * s * s)) for h in range(3, 8))


def spectral_objective(P: np.ndarray, dt: float, w0: float):
    """J and dJ/dP_n for the samples P_n, n = 0..T (spectral weight of the Fourier transform
    of P(t), Sec. "SVD acceleration of TD-aGW"; window as in harmonic_window)."""
    n = np.arange(P.size)
    w = 2 * np.pi * np.arange(P.size) / (P.size * dt)
    E = np.exp(-1j * np.outer(w, n * dt)) * dt          # (freq, time)
    F = E @ P
    wgt = harmonic_window(w, w0)
    J = float(np.sum(wgt * np.abs(F) ** 2))
    dJ = 2.0 * np.real(np.conj(F * wgt) @ E)            # d/dP_n sum wgt |F|^2
    return J, dJ


def _blocks(model, v):
    return v.reshape(model.Nk, model.Nb, model.Nb)


def _herm(a):
    return np.conj(np.swapaxes(a, -1, -2))


def vjp(model, apply_K, apply_KH, E, direction, X, g):
    """(Xbar, Ebar) of the right-hand side of Eq. tdagw, f(X, E) = -i [A(X), rho0 + X], for
    the cotangent g (derivation in the module doc)."""
    Nb = model.Nb
    D = direction[0] * model.dx + direction[1] * model.dy
    A = _blocks(model, apply_K(X)) + E * D
    idx = np.arange(Nb)
    A[:, idx, idx] += model.eps
    rho = _blocks(model, X).copy()
    rho[:, idx, idx] += model.occ
    G = _blocks(model, g)
    Ah, rh = _herm(A), _herm(rho)
    c1 = 1j * (Ah @ G - G @ Ah)
    m = 1j * (G @ rh - rh @ G)
    xbar = c1.reshape(-1) + apply_KH(m.reshape(-1))
    ebar = float(np.real(np.sum(np.conj(G) * (-1j) * (D @ rho - rho @ D))))
    return xbar, ebar


def forward_states(model, apply_K, samples, dt, T, direction):
    """States x_0..x_T and observables of the RK4 run of Eq. tdagw (the oracle forward)."""
    obs, _, states = op.rk4(model, apply_K, samples, dt, T, direction=direction,
                            record_states=True)
    return obs, states


def observable_gradients(model):
    """Gradients of the observables of Sec. "SVD acceleration of TD-aGW" (P_x, J_x, occ_c1)
    with respect to the state X in the real inner product
    <a, b> = Re sum conj(a_i) b_i.  Each observable is Re sum_k sum_nm X_nm O_mn / Nk with O
    Hermitian (d^x, v^x, the projector on c1), so its gradient is O_nm / Nk."""
    occ = np.zeros((model.Nk, model.Nb, model.Nb), dtype=np.complex128)
    occ[:, model.c1, model.c1] = 1.0
    return [o.reshape(-1) / model.Nk for o in (model.dx, model.vx, occ)]


def adjoint(model, apply_K, apply_KH, samples, dt, T, direction, dJdP, dJdJ=None, dJdocc=None):
    """Exact adjoint of the discrete RK4 map of Eq. tdagw: dJ/dE_j for the half-step field
    samples j = 0..2T, given the derivatives of the
    objective with respect to the observables P_x, J_x and occ_c1 at steps n = 0..T (the
    last two optional, zero by default)."""
    _, states = forward_states(model, apply_K, samples, dt, T, direction)
    gP, gJ, go = observable_gradients(model)
    dJdJ = np.zeros(T + 1) if dJdJ is None else np.asarray(dJdJ)
    dJdocc = np.zeros(T + 1) if dJdocc is None else np.asarray(dJdocc)

    def direct(n):
        return dJdP[n] * gP + dJdJ[n] * gJ + dJdocc[n] * go

    h = dt
    lam = direct(T)
    gE = np.zeros(2 * T + 1)

    def f(j, X):
        Ej = samples[j]
        return op.rhs(model, apply_K, Ej * direction[0], Ej * direction[1], X)

    for n in range(T - 1, -1, -1):
        x = states[n]
        k1 = f(2 * n, x)
        X2 = x + 0.5 * h * k1
        k2 = f(2 * n + 1, X2)
        X3 = x + 0.5 * h * k2
        k3 = f(2 * n + 1, X3)
        X4 = x + h * k3
        g4 = h / 6 * lam
        mu4, e4 = vjp(model, apply_K, apply_KH, samples[2 * n + 2], direction, X4, g4)
        g3 = h / 3 * lam + h * mu4
        mu3, e3 = vjp(model, apply_K, apply_KH, samples[2 * n + 1], direction, X3, g3)
        g2 = h / 3 * lam + 0.5 * h * mu3
        mu2, e2 = vjp(model, apply_K, apply_KH, samples[2 * n + 1], direction, X2, g2)
        g1 = h / 6 * lam + 0.5 * h * mu2
        mu1, e1 = vjp(model, apply_K, apply_KH, samples[2 * n], direction, x, g1)
        gE[2 * n] += e1
        gE[2 * n + 1] += e2 + e3
        gE[2 * n + 2] += e4
        lam = lam + mu1 + mu2 + mu3 + mu4 + direct(n)
    return gE


def pulse_param_jacobian(pulse, dt: float, T: int) -> np.ndarray:
    """dE_j / d(E0, omega, t0, sigma) for the Gaussian * cos pulse of Sec. "SVD acceleration
    of TD-aGW"; shape (2T+1, 4)."""
    t = 0.5 * dt * np.arange(2 * T + 1)
    g = np.exp(-((t - pulse.t0) ** 2) / (2 * pulse.sigma ** 2))
    c, s = np.cos(pulse.omega * t), np.sin(pulse.omega * t)
    E = pulse.E0 * g * c
    return np.stack([g * c,
                     -pulse.E0 * g * t * s,
                     E * (t - pulse.t0) / pulse.sigma ** 2,
                     E * (t - pulse.t0) ** 2 / pulse.sigma ** 3], axis=1)


def objective_and_gradients(model, apply_K, apply_KH, pulse, dt, T):
    """J, dJ/d(E0, omega, t0, sigma) and dJ/dE_j for one trajectory of Eq. tdagw driven by the
    Gaussian * cos pulse of Sec. "SVD acceleration of TD-aGW"."""
    direction = (pulse.dir_x, pulse.dir_y)
    samples = op.half_step_samples(pulse, dt, T)
    obs, _ = op.rk4(model, apply_K, samples, dt, T, direction=direction)
    J, dJdP = spectral_objective(obs[:, 0], dt, pulse.omega)
    gE = adjoint(model, apply_K, apply_KH, samples, dt, T, direction, dJdP)
    gp = pulse_param_jacobian(pulse, dt, T).T @ gE
    return J, gp, gE
