"""High-harmonic spectrum of a recorded current (FP64).

Test infrastructure only (see the package header).

Sec. "SVD acceleration of TD-aGW": HHG(w) = | w int J(t) e^{-i w t} dt |^2 with
J(t) = Tr(rho(t) v).  Readings: the time integral over the recorded steps t_n = n dt,
n = 0 .. T, by the rectangle rule (the recorded current starts at J(0) = 0); J is the
x-component of the current (the velocity operator along x), for any field direction of an
angle sweep (Appendix C).
"""
from __future__ import annotations

import numpy as np


def hhg_spectrum(J: np.ndarray, dt: float, omega: np.ndarray) -> np.ndarray:
    """HHG(w) of Sec. "SVD acceleration of TD-aGW" (and Appendix C):
    | w sum_n J(t_n) e^{-i w t_n} dt |^2 for each w in omega; J of length T + 1."""
    J = np.asarray(J, dtype=np.float64)
    omega = np.asarray(omega, dtype=np.float64)
    t = np.arange(J.size) * dt
    F = np.exp(-1j * np.outer(omega, t)) @ J * dt
    return np.abs(omega * F) ** 2


def harmonic_grid(omega0: float, max_order: float, n: int) -> np.ndarray:
    """n frequencies evenly spaced on (0, max_order * omega0] (spectra in harmonic orders of
    the driving frequency, Fig. svd_time_freq, Appendix C)."""
    return omega0 * max_order * np.arange(1, n + 1) / n
