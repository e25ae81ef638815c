"""Planted mistakes in the oracle must trip at least one pin (CPU only).

Each case patches one plausible slip into a copy of an oracle function — a transposed
overlap, a dropped commutator term, a wrong sign — and checks that the pin built for it
fails.  This guards the pins themselves.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import kernel as ok
from oracle import model as om
from oracle import propagate as op


@pytest.fixture(scope="module")
def m4():
    return om.Model(wl.small_model(4, 2))


def _kernel_transposed_hole(model):
    """Slip: (U_k^+ U_k')_{m m'} instead of (U_k'^+ U_k)_{m' m} in the hole factor."""
    p, Nk, Nb = model.p, model.Nk, model.Nb
    W = ok.W_matrix(p)
    O = np.einsum("kin,qip->kqnp", model.U.conj(), model.U)
    K = -W[:, :, None, None, None, None] * O[:, :, :, None, :, None] * O[:, :, None, :, None, :]
    return np.transpose(K, (0, 2, 3, 1, 4, 5)).reshape(Nk * Nb * Nb, Nk * Nb * Nb)


def test_transposed_hole_overlap_breaks_gauge_covariance(m4):
    rng = np.random.default_rng(11)
    ph = rng.uniform(0, 2 * np.pi, (m4.Nk, m4.Nb))
    K1, K2 = _kernel_transposed_hole(m4), _kernel_transposed_hole(m4.rephased(ph))
    e = np.exp(1j * ph)
    pair = (e.conj()[:, :, None] * e[:, None, :]).reshape(-1)
    assert np.abs(K2 - pair[:, None] * K1 * pair.conj()[None, :]).max() > 1e-6


def test_transposed_hole_overlap_breaks_fft_identity(m4):
    x = wl.random_state(m4.N, 3)
    a, b = _kernel_transposed_hole(m4) @ x, ok.apply_fft(m4, x)
    assert np.abs(a - b).max() > 1e-3 * np.abs(b).max()


def test_wrong_commutator_sign_breaks_rabi(monkeypatch):
    p = wl.small_model(1, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    good = op.rhs

    def bad_rhs(model, apply_K, Ex, Ey, X):
        return -good(model, apply_K, Ex, Ey, X).conj()   # i[H, rho] instead of -i[H, rho] (conj flips i)
    monkeypatch.setattr(op, "rhs", bad_rhs)
    import scipy.linalg
    E, Ttot, dt = 0.01, 40.0, 0.2
    T = int(Ttot / dt)
    _, x = op.rk4(mdl, lambda v: K @ v, op.half_step_samples(wl.Pulse(E0=E, kind=1), dt, T), dt, T)
    W0 = -K[0, 0].real
    rho0 = mdl.rho0()[0]
    Ut = scipy.linalg.expm(-1j * (np.diag(mdl.eps[0]) + E * mdl.dx[0] + W0 * rho0) * Ttot)
    exact = Ut @ rho0 @ Ut.conj().T
    assert np.abs(rho0 + x.reshape(2, 2) - exact).max() > 1e-4


def test_dropped_kernel_term_breaks_rabi():
    """Without dSigma the Rabi frequency misses the W0 rho0 shift."""
    p = wl.small_model(1, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    import scipy.linalg
    E, Ttot, dt = 0.01, 40.0, 0.2
    T = int(Ttot / dt)
    _, x = op.rk4(mdl, lambda v: 0 * v, op.half_step_samples(wl.Pulse(E0=E, kind=1), dt, T), dt, T)
    W0 = -K[0, 0].real
    rho0 = mdl.rho0()[0]
    Ut = scipy.linalg.expm(-1j * (np.diag(mdl.eps[0]) + E * mdl.dx[0] + W0 * rho0) * Ttot)
    exact = Ut @ rho0 @ Ut.conj().T
    assert np.abs(rho0 + x.reshape(2, 2) - exact).max() > 1e-4


def test_wrong_W0_breaks_quadrature_pin():
    import scipy.integrate
    p = wl.small_model(12, 1)
    A = p.Nk * p.a ** 2
    h = np.pi / (p.L * p.a)
    f = lambda y, x: ok.coulomb_W(np.hypot(x, y), A, p.r0)
    v, _ = scipy.integrate.dblquad(f, 0, h, lambda x: 0.0, lambda x: x, epsabs=0, epsrel=1e-12)
    brute = 8.0 * v / (4.0 * h * h)
    # slip: average over the disc of radius h instead of the square
    disc = (2 * np.pi / (A * p.r0)) * 2 * np.pi * np.log1p(p.r0 * h) / (np.pi * h * h)
    assert abs(disc - brute) / brute > 1e-3


def test_swapped_channel_breaks_full_rank_reconstruction(monkeypatch):
    """Slip: the channel block read with p and q exchanged (rows of pair q, columns of pair
    p).  The full-rank channel-wise kernel then differs from K."""
    from oracle import channel as oc
    m = om.Model(wl.small_model(4, 1))
    K = ok.dense_kernel(m)
    P = m.Nb * m.Nb
    monkeypatch.setattr(oc, "channel_block", lambda A, Nb, p, q: A[q::P, p::P].copy())
    D, U, S, V = oc.channel_svd(K, m.Nb, m.Nk)
    assert np.abs(oc.assemble(D, U, S, V) - K).max() > 1e-6 * np.abs(K).max()


def test_unconjugated_v_breaks_channel_apply_pin():
    """Slip: V^T instead of V^H in the channel apply; the dense kernel of the same factors
    disagrees with it."""
    from oracle import channel as oc
    m = om.Model(wl.small_model(4, 1))
    K = ok.dense_kernel(m)
    D, U, S, V = oc.channel_svd(K, m.Nb, 6)
    x = wl.random_state(m.N, 4)
    P, Nk = m.Nb * m.Nb, m.Nk
    xs = x.reshape(Nk, P)
    bad = np.zeros((Nk, P), complex)
    for p in range(P):
        bad[:, p] = D[p] @ xs[:, p]
        for q in range(P):
            if q != p:
                bad[:, p] += U[p, q] @ (S[p, q] * (V[p, q].T @ xs[:, q]))
    good = oc.assemble(D, U, S, V) @ x
    assert np.abs(bad.reshape(-1) - good).max() > 1e-6 * np.abs(good).max()


def test_exchange_orbitals_at_one_site_break_rank_pin(monkeypatch):
    """Slip: both orbitals of a copy placed at the cell origin (no exp(i G . tau) phase).
    Every shell then gives the same matrix elements and K^x drops to rank 1."""
    import dataclasses

    import scipy.linalg
    m = om.Model(dataclasses.replace(wl.small_model(4, 1), exchange=1.0))
    M, v = ok.exchange_vectors(m)
    Mbad = np.broadcast_to(np.einsum("kon,kom->knm", m.U.conj(), m.U)[:, None], M.shape)
    monkeypatch.setattr(ok, "exchange_vectors", lambda model: (Mbad, v))
    ev = np.abs(scipy.linalg.eigvalsh(ok.exchange_kernel(m)))
    assert (ev > 1e-12 * ev.max()).sum() != 2


def test_field_samples_shifted_half_step_break_commuting_closed_form(monkeypatch):
    """Slip: stage samples taken half a step early (E((j - 1) dt / 2)): the time-dependent
    commuting closed form then converges at first order only."""
    import copy
    import scipy.integrate
    import scipy.linalg

    def shifted(pulse, dt, T):
        return np.array([op.field_value(pulse, 0.5 * (j - 1) * dt) for j in range(2 * T + 1)])
    monkeypatch.setattr(op, "half_step_samples", shifted)
    mdl = om.Model(wl.small_model(3, 1))
    m0 = copy.copy(mdl)
    m0.eps = np.zeros_like(mdl.eps)
    pulse = wl.Pulse(E0=0.05, omega=0.3, t0=8.0, sigma=3.0)
    th, Ttot = (0.6, 0.8), 16.0
    A = scipy.integrate.quad(lambda t: op.field_value(pulse, t), 0.0, Ttot, epsabs=1e-14, limit=200)[0]
    rho0 = mdl.rho0()
    D = th[0] * mdl.dx + th[1] * mdl.dy
    exact = np.array([scipy.linalg.expm(-1j * A * D[k]) @ rho0[k] @ scipy.linalg.expm(1j * A * D[k])
                      for k in range(mdl.Nk)])
    errs = []
    for dt in (0.4, 0.2, 0.1):
        T = int(round(Ttot / dt))
        _, x = op.rk4(m0, lambda v: np.zeros_like(v), op.half_step_samples(pulse, dt, T), dt, T, direction=th)
        errs.append(np.abs(rho0 + x.reshape(mdl.Nk, mdl.Nb, mdl.Nb) - exact).max())
    assert errs[2] > 1e-9 or not all(12.0 < a / b < 20.0 for a, b in zip(errs, errs[1:]))
    assert errs[0] / errs[1] < 4.0


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")  # the slip oscillates fast
@pytest.mark.parametrize("slip", ["envelope_product", "cos_carrier"])
def test_garbled_strong_field_pulse_breaks_area_pin(monkeypatch, slip):
    """Slips in the sin^2-envelope pulse: the printed sin^2(pi t T_pulse) taken literally, or
    a cos carrier; either misses the closed-form pulse area."""
    import scipy.integrate
    good = op.field_value

    def bad(pulse, t):
        if pulse.kind != 2:
            return good(pulse, t)
        if t < 0.0 or t > pulse.T_pulse:
            return 0.0
        if slip == "envelope_product":
            return pulse.E0 * np.sin(np.pi * t * pulse.T_pulse) ** 2 * np.sin(pulse.omega * t)
        return pulse.E0 * np.sin(np.pi * t / pulse.T_pulse) ** 2 * np.cos(pulse.omega * t)
    monkeypatch.setattr(op, "field_value", bad)
    w, T = 0.13, 250.0
    p = wl.Pulse(E0=0.01, omega=w, T_pulse=T, kind=2)
    q = scipy.integrate.quad(lambda t: op.field_value(p, t), 0.0, T, limit=400, epsabs=1e-14)[0]
    a = np.pi / T
    area = 2 * a * a * p.E0 * (1 - np.cos(w * T)) / (w * (4 * a * a - w * w))
    assert abs(q - area) > 1e-3 * abs(area)


@pytest.mark.parametrize("slip", ["sigma_squared", "no_shift", "sin_carrier"])
def test_garbled_gaussian_pulse_breaks_area_pin(monkeypatch, slip):
    """Slips in the Gaussian * cos pulse (width sigma^2 instead of 2 sigma^2, carrier on
    t - t0, sine carrier) miss the Fourier-transform area."""
    import scipy.integrate
    good = op.field_value

    def bad(pulse, t):
        if pulse.kind != 0:
            return good(pulse, t)
        env = np.exp(-((t - pulse.t0) ** 2) / ((1.0 if slip == "sigma_squared" else 2.0) * pulse.sigma ** 2))
        if slip == "no_shift":
            return pulse.E0 * env * np.cos(pulse.omega * (t - pulse.t0))
        if slip == "sin_carrier":
            return pulse.E0 * env * np.sin(pulse.omega * t)
        return pulse.E0 * env * np.cos(pulse.omega * t)
    monkeypatch.setattr(op, "field_value", bad)
    w, sigma, t0 = 0.1, 5.0, 60.0
    p = wl.Pulse(E0=0.01, omega=w, t0=t0, sigma=sigma, kind=0)
    q = scipy.integrate.quad(lambda t: op.field_value(p, t), 0.0, t0 + 14 * sigma, limit=800,
                             epsabs=1e-16, points=[t0])[0]
    want = p.E0 * sigma * np.sqrt(2 * np.pi) * np.exp(-(w * sigma) ** 2 / 2) * np.cos(w * t0)
    assert abs(q - want) > 1e-3 * abs(want)


def test_unconjugated_bra_in_velocity_breaks_heisenberg_pin():
    """Slip: <u_n| taken without complex conjugation in the band-basis velocity."""
    p = wl.small_model(5, 1)
    mdl = om.Model(p)
    v = np.einsum("kin,kij,kjm->knm", mdl.U, om.dh_dk(mdl.k, p, 0), mdl.U)
    want = 1j * (mdl.eps[:, :, None] - mdl.eps[:, None, :]) * mdl.dx
    off = ~np.eye(mdl.Nb, dtype=bool)
    assert np.abs(v[:, off] - want[:, off]).max() > 1e-3


def _W_slipped(slip):
    """A copy of W_of_offsets with one plausible slip planted."""
    good_W0 = ok.cell_average_W0

    def W(di, dj, p):
        L, a = p.L, p.a
        A = (a * a) if slip == "area_a2" else p.Nk * a * a
        step = 2.0 * np.pi / L if slip == "q_without_a" else 2.0 * np.pi / (L * a)
        q = np.hypot(di * step, dj * step)
        out = np.empty_like(q)
        nz = q > 0
        if slip == "screening_over_r0":
            out[nz] = 2.0 * np.pi / (A * q[nz] * (1.0 + q[nz] / p.r0))
        elif slip == "no_two_pi":
            out[nz] = 1.0 / (A * q[nz] * (1.0 + p.r0 * q[nz]))
        else:
            out[nz] = 2.0 * np.pi / (A * q[nz] * (1.0 + p.r0 * q[nz]))
        out[~nz] = good_W0(np.pi / (L * a), A, p.r0)
        return out
    return W


@pytest.mark.parametrize("slip", ["area_a2", "q_without_a", "screening_over_r0", "no_two_pi"])
def test_slipped_W_breaks_brillouin_zone_pin(monkeypatch, slip):
    """Slips in W(q != 0): the area a^2 instead of Nk a^2, the q spacing 2 pi / L without the
    lattice constant, the screening factor (1 + |q| / r0), a dropped 2 pi.  Each misses the
    Brillouin-zone integral of the Rytova-Keldysh interaction."""
    import test_oracle_pins as pins
    monkeypatch.setattr(ok, "W_of_offsets", _W_slipped(slip))
    raw, rich = pins.bz_sum_errors(Ls=(48, 96, 192))
    assert np.abs(rich).max() > 1e-2 or np.abs(raw[:, -1]).max() > 1e-1


@pytest.mark.parametrize("slip", ["over_N", "over_Nk_Nb", "plain_sum"])
def test_wrong_observables_normalisation_breaks_pin(monkeypatch, slip):
    """Slips in the k-sum normalisation of P, J and occupation: 1/N, 1/(Nk Nb), no 1/Nk."""
    import test_oracle_pins as pins
    good = op.observables

    def bad(model, X):
        o = good(model, X)
        scale = {"over_N": 1.0 / (model.Nb * model.Nb), "over_Nk_Nb": 1.0 / model.Nb,
                 "plain_sum": float(model.Nk)}[slip]
        return o * scale
    monkeypatch.setattr(op, "observables", bad)
    assert pins.observables_normalisation_errors() > 1e-3
