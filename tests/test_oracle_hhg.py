"""Pins of the HHG oracle against the FFT, a closed form and scaling.  No GPU."""
import numpy as np

from oracle import hhg


def test_matches_fft_bins():
    """At the DFT frequencies w_k = 2 pi k / (M dt) the sum is numpy's FFT bin k."""
    rng = np.random.default_rng(4)
    M, dt = 257, 0.2
    J = rng.standard_normal(M)
    k = np.arange(1, 40)
    w = 2 * np.pi * k / (M * dt)
    want = np.abs(w * dt * np.fft.fft(J)[k]) ** 2
    np.testing.assert_allclose(hhg.hhg_spectrum(J, dt, w), want, rtol=1e-11)


def test_single_harmonic_closed_form():
    """J = cos(w0 t) over a whole number of periods: at w0 the sum is M / 2 (discrete
    orthogonality), at the other DFT frequencies zero."""
    M, dt, m = 400, 0.2, 7
    w0 = 2 * np.pi * m / (M * dt)
    J = np.cos(w0 * dt * np.arange(M))
    s = hhg.hhg_spectrum(J, dt, np.array([w0, 2 * w0, 3 * w0]))
    np.testing.assert_allclose(s[0], (w0 * dt * M / 2) ** 2, rtol=1e-12)
    assert s[1] < 1e-20 * s[0] and s[2] < 1e-20 * s[0]


def test_quadratic_in_amplitude_and_time_shift_invariant():
    """HHG(a J) = a^2 HHG(J); delaying J by one step (a current that has ended: J[-1] = 0)
    multiplies the amplitude by the phase e^{-i w dt} and leaves the spectrum unchanged."""
    rng = np.random.default_rng(5)
    J = np.concatenate([rng.standard_normal(99), [0.0]])
    w = np.linspace(0.05, 2.0, 17)
    s = hhg.hhg_spectrum(J, 0.1, w)
    np.testing.assert_allclose(hhg.hhg_spectrum(3 * J, 0.1, w), 9 * s, rtol=1e-12)
    shifted = np.concatenate([[0.0], J[:-1]])
    np.testing.assert_allclose(hhg.hhg_spectrum(shifted, 0.1, w), s, rtol=1e-11)
