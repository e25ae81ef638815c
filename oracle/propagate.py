"""TD-aGW equation of motion, classical RK4 and observables (FP64).

Test infrastructure only (see the package header).

Eq. tdagw: i d/dt rho_k = [H^QP_k + dSigma_k(t) - e E(t).r_k, rho_k], one k index (dipole
approximation).  Readings:
  * The propagated state is drho = rho - rho0 with rho0 = diag(occupations), so
        d drho / dt = -i [H_k(t), rho0_k + drho_k],
        H_k(t) = diag(eps_k) + E(t).d_k + dSigma_k,   dSigma = K . drho.
    The field couples as +E(t).d (the sign -e with e = -1 absorbed; only the relative
    sign of the field matters for the tests, which drive both sides with the same E).
  * The Hamiltonian is "updated at each time step" (Sec. "SVD acceleration"): with RK4
    dSigma is re-evaluated at every stage, the consistent RK4 of the ODE.
  * Classical 4-stage RK4 with stage times t_n, t_n + dt/2, t_n + dt/2, t_n + dt.
  * Observables at every step n = 0..T (t = n dt):
        P_x = (1/Nk) sum_k Re Tr(rho_k d^x_k)          (Sec. "SVD acceleration": A(w) from P(t))
        J_x = (1/Nk) sum_k Re Tr(rho_k v^x_k)          (J = Tr(rho v))
        occ = (1/Nk) sum_k Re rho_{c1 c1 k}             (Fig. svd_time_freq caption)
  * Pulses: kind 0 is E0 exp(-(t - t0)^2 / (2 sigma^2)) cos(w t); kind 1 a constant E0;
    kind 2 the strong-field pulse E0 sin^2(pi t / T_pulse) sin(w t) on [0, T_pulse] (the
    printed "sin^2(pi t T_pulse)" is read as pi t / T_pulse).
"""
from __future__ import annotations

import numpy as np


def field_value(pulse, t: float) -> float:
    """Scalar amplitude E(t) of the pulses of Sec. "SVD acceleration of TD-aGW" (direction
    handled separately)."""
    if pulse.kind == 0:
        return pulse.E0 * np.exp(-((t - pulse.t0) ** 2) / (2.0 * pulse.sigma ** 2)) * np.cos(pulse.omega * t)
    if pulse.kind == 1:
        return pulse.E0
    if pulse.kind == 2:
        if t < 0.0 or t > pulse.T_pulse:
            return 0.0
        return pulse.E0 * np.sin(np.pi * t / pulse.T_pulse) ** 2 * np.sin(pulse.omega * t)
    raise ValueError(f"unknown pulse kind {pulse.kind}")


def half_step_samples(pulse, dt: float, T: int) -> np.ndarray:
    """E(n dt / 2) for n = 0..2T: every RK4 stage time of a T-step run of Eq. tdagw."""
    return np.array([field_value(pulse, 0.5 * j * dt) for j in range(2 * T + 1)])


def rhs(model, apply_K, Ex: float, Ey: float, X: np.ndarray) -> np.ndarray:
    """Right-hand side of Eq. tdagw with dSigma of Eq. sigma-from-k:
    -i [diag(eps) + Ex d^x + Ey d^y + (K X), rho0 + X] per k, flattened like X."""
    Nk, Nb = model.Nk, model.Nb
    Xk = X.reshape(Nk, Nb, Nb)
    dS = apply_K(X).reshape(Nk, Nb, Nb)
    H = dS + Ex * model.dx + Ey * model.dy
    idx = np.arange(Nb)
    H[:, idx, idx] += model.eps
    rho = Xk.copy()
    rho[:, idx, idx] += model.occ
    return (-1j * (H @ rho - rho @ H)).reshape(-1)


def observables(model, X: np.ndarray) -> np.ndarray:
    """(P_x, J_x, occ_c1) of the state rho0 + X: the polarization and current of Sec. "SVD
    acceleration of TD-aGW" and the conduction occupation of Fig. svd_time_freq."""
    rho = model.rho0() + X.reshape(model.Nk, model.Nb, model.Nb)
    P = np.sum(rho * np.swapaxes(model.dx, 1, 2)).real / model.Nk     # sum_nm rho_nm d_mn
    J = np.sum(rho * np.swapaxes(model.vx, 1, 2)).real / model.Nk
    occ = rho[:, model.c1, model.c1].real.mean()
    return np.array([P, J, occ])


def rk4(model, apply_K, samples: np.ndarray, dt: float, T: int, direction=(1.0, 0.0),
        x0: np.ndarray | None = None, record_states: bool = False):
    """T classical RK4 steps of Eq. tdagw from drho = x0 (default 0).

    samples[j] = E(j dt / 2), j = 0..2T (see half_step_samples); the two middle stages
    of a step share the sample at t_n + dt/2.  Returns (obs (T+1, 3), final state) and,
    with record_states, the list of states after each step.
    """
    dxr, dyr = direction
    x = np.zeros(model.N, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    obs = np.empty((T + 1, 3))
    obs[0] = observables(model, x)
    states = [x.copy()] if record_states else None

    def f(j, X):
        E = samples[j]
        return rhs(model, apply_K, E * dxr, E * dyr, X)

    for n in range(T):
        k1 = f(2 * n, x)
        k2 = f(2 * n + 1, x + 0.5 * dt * k1)
        k3 = f(2 * n + 1, x + 0.5 * dt * k2)
        k4 = f(2 * n + 2, x + dt * k3)
        x = x + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        obs[n + 1] = observables(model, x)
        if record_states:
            states.append(x.copy())
    if record_states:
        return obs, x, states
    return obs, x


def rel_l2(a: np.ndarray, b: np.ndarray) -> float:
    """||a - b||_2 / ||b||_2: the relative error of P(t) (Sec. "SVD acceleration of TD-aGW"
    compares spectra; every comparison here uses P(t) itself)."""
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b))
