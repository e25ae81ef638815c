"""Pins of the FP64 oracle against closed forms, invariants and independent routines.

Each test fixes a part of the oracle with something other than the oracle itself, so
that a dropped term, a wrong sign or index, or a transposed operand fails one of them.
No GPU.
"""
import dataclasses

import numpy as np
import pytest
import scipy.integrate
import scipy.linalg

import workloads as wl
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om
from oracle import propagate as op


@pytest.fixture(scope="module")
def m2():
    return om.Model(wl.small_model(6, 1))


@pytest.fixture(scope="module")
def m4():
    return om.Model(wl.small_model(4, 2))


# ---------------------------------------------------------------- model -------------

@pytest.mark.parametrize("nc", [1, 2])
def test_eigenpairs_closed_form(nc):
    """Eigenvalues are off_c +- |d(k)| (textbook 2x2); eigenvectors diagonalise h."""
    p = wl.small_model(5, nc)
    k = om.kgrid(p.L, p.a) + 0.013
    eps, U = om.eigensystem(k, p)
    kx, ky = k[:, 0] * p.a, k[:, 1] * p.a
    d = np.sqrt((p.t * np.sin(kx)) ** 2 + (p.t * np.sin(ky)) ** 2
                + (p.Delta + p.m * (2 - np.cos(kx) - np.cos(ky))) ** 2)
    want = np.sort(np.concatenate([np.stack([p.offsets[c] - d, p.offsets[c] + d], 1)
                                   for c in range(nc)], 1), axis=1)
    np.testing.assert_allclose(eps, want, atol=1e-14)
    H = om.h_orbital(k, p)
    np.testing.assert_allclose(H @ U, U * eps[:, None, :], atol=1e-14)
    # gauge rule: largest-modulus component real and positive
    idx = np.argmax(np.abs(U), axis=1)
    piv = np.take_along_axis(U, idx[:, None, :], axis=1)
    assert np.all(piv.real > 0) and np.abs(piv.imag).max() < 1e-15


def test_dh_dk_matches_numerical_derivative():
    p = wl.small_model(3, 2)
    k = om.kgrid(p.L, p.a) + 0.02
    for ax in (0, 1):
        e = np.zeros(2)
        e[ax] = 1e-6
        num = (om.h_orbital(k + e, p) - om.h_orbital(k - e, p)) / 2e-6
        np.testing.assert_allclose(om.dh_dk(k, p, ax), num, atol=1e-8)


@pytest.mark.parametrize("nc", [1, 2])
def test_dipole_matches_interband_formula(nc):
    """i<n|du_m> = i <n|dh|m> / (eps_m - eps_n) for n != m; diagonal zero after transport."""
    p = wl.small_model(5, nc)
    mdl = om.Model(p)
    for ax, d in ((0, mdl.dx), (1, mdl.dy)):
        dh = np.einsum("kin,kij,kjm->knm", mdl.U.conj(), om.dh_dk(mdl.k, p, ax), mdl.U)
        de = mdl.eps[:, None, :] - mdl.eps[:, :, None]          # eps_m - eps_n
        off = ~np.eye(p.Nb, dtype=bool)
        want = np.zeros_like(dh)
        want[:, off] = 1j * dh[:, off] / de[:, off]
        np.testing.assert_allclose(d, want, atol=2e-8)
        assert np.abs(np.diagonal(d, axis1=1, axis2=2)).max() < 1e-9
        np.testing.assert_allclose(d, np.conj(np.swapaxes(d, 1, 2)), atol=1e-15)


def test_velocity_diagonal_is_band_slope(m4):
    """Hellmann-Feynman: v_nn = d eps_n / dk_x (central difference of eigenvalues)."""
    p = m4.p
    e = np.array([1e-6, 0.0])
    slope = (om.eigensystem(m4.k + e, p)[0] - om.eigensystem(m4.k - e, p)[0]) / 2e-6
    np.testing.assert_allclose(np.diagonal(m4.vx, axis1=1, axis2=2).real, slope, atol=1e-8)


@pytest.mark.parametrize("nc", [1, 2])
def test_velocity_is_commutator_with_position(nc):
    """Heisenberg relation v = i [H, r] in the band basis: v_nm = i (eps_n - eps_m) d_nm for
    n != m, with d the finite-difference Berry dipole (computed independently of the
    analytic velocity); v Hermitian."""
    mdl = om.Model(wl.small_model(5, nc))
    v, d, eps = mdl.vx, mdl.dx, mdl.eps
    want = 1j * (eps[:, :, None] - eps[:, None, :]) * d
    off = ~np.eye(mdl.Nb, dtype=bool)
    assert np.abs(v[:, off]).max() > 0.1
    np.testing.assert_allclose(v[:, off], want[:, off], atol=2e-8)
    np.testing.assert_allclose(v, np.conj(np.swapaxes(v, 1, 2)), atol=1e-15)


def test_four_band_copies_decouple(m4):
    """Bands of different copies have zero overlap, dipole and velocity."""
    # bands 0, 2 are copy 0 (lower/upper); 1, 3 are copy 1 (offset 0.03)
    U = m4.U
    w0 = np.abs(U[:, 0:2, :]) ** 2
    copy = (w0.sum(axis=1) < 0.5).astype(int)                  # (Nk, Nb)
    assert np.all(copy == np.array([0, 1, 0, 1]))
    for X in (m4.dx, m4.dy, m4.vx):
        cross = X[:, copy[0][:, None] != copy[0][None, :]]
        assert np.abs(cross).max() < 1e-9


# ---------------------------------------------------------------- W(q) ---------------

def test_cell_average_against_2d_quadrature():
    """W0 = mean of W over the mini-cell, checked by adaptive Cartesian 2D quadrature."""
    p = wl.small_model(12, 1)
    A = p.Nk * p.a ** 2
    h = np.pi / (p.L * p.a)
    f = lambda y, x: ok.coulomb_W(np.hypot(x, y), A, p.r0)
    # quarter square [0,h]^2 (W is even in qx, qy); split the integrable corner singularity
    val1, _ = scipy.integrate.dblquad(f, 0, h, lambda x: 0.0, lambda x: x, epsabs=0, epsrel=1e-12)
    brute = 8.0 * val1 / (4.0 * h * h)
    assert abs(ok.cell_average_W0(h, A, p.r0) - brute) / brute < 1e-9


def test_cell_average_unscreened_limit():
    """r0 -> 0: mean of 1/|q| over the square of half-side h is 2 ln(1 + sqrt 2) / h."""
    A, h = 3.7, 0.05
    got = ok.cell_average_W0(h, A, 1e-10)
    want = (2 * np.pi / A) * 2 * np.log1p(np.sqrt(2.0)) / h
    assert abs(got - want) / want < 1e-8


def bz_lattice_sum(L, R, r0=20.0, a=6.0):
    """sum_q W(q) cos(q . R) over the L x L grid with the oracle's W (W0 at q = 0)."""
    p = dataclasses.replace(wl.small_model(L, 1), r0=r0, a=a)
    di = ok.min_image(np.arange(L), L)
    DI, DJ = np.meshgrid(di, di, indexing="ij")
    W = ok.W_of_offsets(DI, DJ, p)
    dq = 2 * np.pi / (L * a)
    return float(np.sum(W * np.cos(dq * (DI * R[0] + DJ * R[1]))))


def bz_continuum(R, r0=20.0, a=6.0):
    """int over the square Brillouin zone |qx|,|qy| <= pi/a of d^2q/(2 pi)^2 of the 2D
    Rytova-Keldysh interaction 2 pi / (|q| (1 + r0 |q|)) times cos(q . R), by adaptive
    quadrature in polar coordinates (the 1/|q| singularity cancels against the Jacobian)."""
    qm = np.pi / a
    rmax = lambda th: qm / max(abs(np.cos(th)), abs(np.sin(th)))
    f = lambda q, th: np.cos(q * (np.cos(th) * R[0] + np.sin(th) * R[1])) / (2 * np.pi * (1 + r0 * q))
    edges = [k * np.pi / 4 for k in range(9)]                  # split at the square's corners
    return sum(scipy.integrate.dblquad(f, t0, t1, lambda th: 0.0, rmax, epsabs=1e-13, epsrel=1e-11)[0]
               for t0, t1 in zip(edges, edges[1:]))


BZ_R = [(0.0, 0.0), (6.0, 0.0), (12.0, 0.0), (6.0, 6.0), (30.0, 0.0)]


def bz_sum_errors(Ls=(96, 192, 384)):
    """Relative deviation of the lattice sums from the continuum integral, per R and L, and
    of the Richardson extrapolation 2 s(L_max) - s(L_max / 2)."""
    raw, rich = [], []
    for R in BZ_R:
        c = bz_continuum(R)
        s = [bz_lattice_sum(L, R) for L in Ls]
        raw.append([(x - c) / c for x in s])
        rich.append((2 * s[-1] - s[-2] - c) / c)
    return np.array(raw), np.array(rich)


def test_W_lattice_sum_converges_to_brillouin_zone_integral():
    """W(q) at q != 0 (Eq. bse-direct-def with the Rytova-Keldysh screening of Appendix B):
    with the Born-von Karman area A = Nk a^2 the sum over the k-grid of W(q) e^{iq.R} is a
    Riemann sum of the continuum integral over the Brillouin zone (spacing 2 pi / (L a),
    cell area (2 pi)^2 / A), so it must converge to that integral, computed here by adaptive
    quadrature, with an error falling as 1/L at every lattice vector R.  A wrong area
    (a^2), screening factor (1 + |q| / r0), prefactor or q spacing misses the integral by
    a factor, whatever the grid."""
    raw, rich = bz_sum_errors()
    assert np.abs(raw[:, -1]).max() < 1e-2, raw
    ratio = raw[:, 1] / raw[:, 2]
    assert np.all((ratio > 1.8) & (ratio < 2.2)), ratio       # first order in 1/L
    assert np.abs(rich).max() < 2e-4, rich


def test_W_real_space_tail_is_rytova_keldysh():
    """Far from the origin the potential of 2 pi / (|q| (1 + r0 |q|)) is the Rytova-Keldysh
    form (pi / (2 r0)) [H0(R / r0) - Y0(R / r0)] (Struve H0, Neumann Y0; the 2D Fourier
    transform of the interaction).  Leaving out |q| > pi/a changes it by a share that decays
    with R, so at R = 10 a .. 30 a both the Brillouin-zone integral and the oracle's lattice
    sums (extrapolated from L = 384, 768) must land on the closed form: this ties the
    oracle's q-grid scale and prefactors to real-space distance without any quadrature."""
    import scipy.special
    r0, a = 20.0, 6.0
    for n in (10, 20, 30):
        R = (n * a, 0.0)
        want = np.pi / (2 * r0) * (scipy.special.struve(0, R[0] / r0) - scipy.special.y0(R[0] / r0))
        s1, s2 = bz_lattice_sum(384, R), bz_lattice_sum(768, R)
        assert abs(2 * s2 - s1 - want) < 3e-3 * want, (n, 2 * s2 - s1, want)
        assert abs(bz_continuum(R) - want) < 3e-3 * want


# ---------------------------------------------------------------- kernel -------------

@pytest.mark.parametrize("name", ["m2", "m4"])
def test_kernel_hermitian_and_diag(name, request):
    mdl = request.getfixturevalue(name)
    K = ok.dense_kernel(mdl)
    assert np.abs(K - K.conj().T).max() == 0.0
    W0 = ok.cell_average_W0(np.pi / (mdl.p.L * mdl.p.a), mdl.Nk * mdl.p.a ** 2, mdl.p.r0)
    np.testing.assert_allclose(np.diag(K), -W0, rtol=1e-14)
    np.testing.assert_allclose(ok.kernel_diag(mdl), np.diag(K), rtol=1e-14)


@pytest.mark.parametrize("name", ["m2", "m4"])
def test_kernel_dense_equals_fft_convolution(name, request):
    """Dense K.x == the independent FFT-convolution form, to rounding."""
    mdl = request.getfixturevalue(name)
    K = ok.dense_kernel(mdl)
    x = wl.random_state(mdl.N, 3)
    a, b = ok.apply_dense(K, x), ok.apply_fft(mdl, x)
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()


def test_kernel_entries_by_scalar_loops(m4):
    """Sampled entries and rows of the dense matrix against the entry formula."""
    K = ok.dense_kernel(m4)
    rng = np.random.default_rng(7)
    for _ in range(50):
        r, c = rng.integers(0, m4.N, 2)
        assert abs(K[r, c] - ok.kernel_entry(m4, int(r), int(c))) < 1e-16
    for r in rng.integers(0, m4.N, 5):
        np.testing.assert_allclose(ok.kernel_row(m4, int(r)), K[r], atol=1e-17)


def test_kernel_gauge_covariance(m4):
    """Rephasing bands multiplies K entries by the matching pair phases (index check)."""
    rng = np.random.default_rng(11)
    ph = rng.uniform(0, 2 * np.pi, (m4.Nk, m4.Nb))
    K1, K2 = ok.dense_kernel(m4), ok.dense_kernel(m4.rephased(ph))
    e = np.exp(1j * ph)
    pair = (e.conj()[:, :, None] * e[:, None, :]).reshape(-1)     # phase of rho_nm,k
    np.testing.assert_allclose(K2, pair[:, None] * K1 * pair.conj()[None, :], atol=1e-16)


def test_single_k_kernel_is_minus_W0_identity():
    p = wl.small_model(1, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    W0 = ok.cell_average_W0(np.pi / p.a, p.a ** 2, p.r0)
    np.testing.assert_allclose(K, -W0 * np.eye(4), atol=1e-15)


# ---------------------------------------------------------------- SVD ----------------

def test_svd_full_rank_and_eckart_young(m2):
    K = ok.dense_kernel(m2)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, m2.N)
    assert np.abs(olr.reconstruct(d, U, S, V) - K).max() < 1e-14 * np.abs(K).max() * m2.N
    sv = olr.singular_values(Koff)
    # Hermitian K^off: singular values are |eigenvalues| (independent LAPACK routine)
    np.testing.assert_allclose(np.sort(np.abs(scipy.linalg.eigvalsh(Koff)))[::-1], sv, atol=1e-15)
    for r in (5, 40, 200):
        U, S, V = olr.truncated_svd(Koff, r)
        err = np.linalg.norm(Koff - (U * S) @ V.conj().T)
        assert abs(err - np.sqrt(np.sum(sv[r:] ** 2))) < 1e-12 * np.linalg.norm(Koff)


def test_lowrank_apply_matches_reconstruction(m2):
    K = ok.dense_kernel(m2)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, 30)
    x = wl.random_state(m2.N, 5)
    np.testing.assert_allclose(olr.apply_lowrank(d, U, S, V, x),
                               olr.reconstruct(d, U, S, V) @ x, atol=1e-16)


def test_r_squared_definition():
    y = np.array([1.0, 2.0, 3.0, 4.0])
    assert olr.r_squared(y, y) == 1.0
    assert abs(olr.r_squared(y, np.full(4, y.mean()))) < 1e-15


# ---------------------------------------------------------------- dynamics -----------

def _rabi_exact(mdl, E, t):
    W0 = -ok.dense_kernel(mdl)[0, 0].real
    rho0 = mdl.rho0()[0]
    Heff = np.diag(mdl.eps[0]) + E * mdl.dx[0] + W0 * rho0
    Ut = scipy.linalg.expm(-1j * Heff * t)
    return Ut @ rho0 @ Ut.conj().T


def test_rabi_closed_form_single_k():
    """Nk = 1, constant field: K = -W0 I, so rho(t) = e^{-iHt} rho0 e^{iHt} with
    H = H0 + E d + W0 rho0 exactly; RK4 error must shrink ~16x when dt halves."""
    p = wl.small_model(1, 1)
    mdl = om.Model(p)
    K = ok.dense_kernel(mdl)
    E = 0.01
    pulse = wl.Pulse(E0=E, kind=1)
    Ttot = 40.0
    errs = []
    for dt in (0.4, 0.2, 0.1):
        T = int(round(Ttot / dt))
        s = op.half_step_samples(pulse, dt, T)
        _, x = op.rk4(mdl, lambda v: K @ v, s, dt, T)
        rho = mdl.rho0()[0] + x.reshape(2, 2)
        errs.append(np.abs(rho - _rabi_exact(mdl, E, Ttot)).max())
    assert errs[1] < 3e-7
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0


def _commuting_field_errors(dts, Ttot=16.0):
    """Degenerate bands (eps = 0) and no kernel: H_k(t) = E(t) d_k with d_k = cos(th) d^x_k +
    sin(th) d^y_k commutes with itself at all times, so rho_k(t) = e^{-i A d_k} rho0 e^{i A d_k}
    with A = int_0^t E (quadrature).  Max |rho - exact| over k at t = Ttot for each dt."""
    import copy
    mdl = om.Model(wl.small_model(3, 1))
    m0 = copy.copy(mdl)
    m0.eps = np.zeros_like(mdl.eps)
    pulse = wl.Pulse(E0=0.05, omega=0.3, t0=8.0, sigma=3.0)
    th = (0.6, 0.8)
    A = scipy.integrate.quad(lambda t: op.field_value(pulse, t), 0.0, Ttot, epsabs=1e-14, limit=200)[0]
    rho0 = mdl.rho0()
    D = th[0] * mdl.dx + th[1] * mdl.dy
    exact = np.array([scipy.linalg.expm(-1j * A * D[k]) @ rho0[k] @ scipy.linalg.expm(1j * A * D[k])
                      for k in range(mdl.Nk)])
    errs = []
    for dt in dts:
        T = int(round(Ttot / dt))
        _, x = op.rk4(m0, lambda v: np.zeros_like(v), op.half_step_samples(pulse, dt, T), dt, T, direction=th)
        errs.append(np.abs(rho0 + x.reshape(mdl.Nk, mdl.Nb, mdl.Nb) - exact).max())
    return errs, np.abs(exact - rho0).max()


def test_time_dependent_field_commuting_closed_form():
    """Pins the field sampling of the RK4 stages (t_n, t_n + dt/2 twice, t_n + dt) and the
    field direction with a time-dependent pulse: fourth-order convergence to the exact
    rotation (a sample misplaced by half a step leaves first order)."""
    errs, moved = _commuting_field_errors((0.4, 0.2, 0.1))
    assert moved > 0.1
    assert errs[2] < 1e-9
    for a, b in zip(errs, errs[1:]):
        assert 12.0 < a / b < 20.0, errs


@pytest.mark.parametrize("w,sigma,t0", [(0.1, 5.0, 60.0), (0.06, 30.0, 320.0), (0.3, 2.0, 25.0)])
def test_gaussian_pulse_area_is_its_fourier_transform(w, sigma, t0):
    """Gaussian * cos pulse: int E dt = E0 sigma sqrt(2 pi) exp(-w^2 sigma^2 / 2) cos(w t0)
    (the Fourier transform of a Gaussian; t0 >= 10 sigma makes the part before t = 0
    negligible).  Fixes the width convention 2 sigma^2, the shift t - t0 and the carrier."""
    p = wl.Pulse(E0=0.01, omega=w, t0=t0, sigma=sigma, kind=0)
    q = scipy.integrate.quad(lambda t: op.field_value(p, t), 0.0, t0 + 14 * sigma, limit=800,
                             epsabs=1e-16, points=[t0])[0]
    want = p.E0 * sigma * np.sqrt(2 * np.pi) * np.exp(-(w * sigma) ** 2 / 2) * np.cos(w * t0)
    assert abs(q - want) < 1e-11 * abs(want)


def _sin2_pulse_area(E0, w, T):
    """int_0^T E0 sin^2(pi t / T) sin(w t) dt by product-to-sum identities (a = pi / T,
    2 a T = 2 pi): 2 a^2 E0 (1 - cos w T) / (w (4 a^2 - w^2))."""
    a = np.pi / T
    return 2 * a * a * E0 * (1 - np.cos(w * T)) / (w * (4 * a * a - w * w))


@pytest.mark.parametrize("w,T", [(0.057, 400.0), (0.13, 250.0), (0.31, 97.3)])
def test_strong_field_pulse_area_closed_form(w, T):
    """The sin^2-envelope pulse (envelope sin^2(pi t / T_pulse) on [0, T_pulse], carrier
    sin(w t)): its time integral against the closed form, and zero outside the window."""
    p = wl.Pulse(E0=0.01, omega=w, T_pulse=T, kind=2)
    q = scipy.integrate.quad(lambda t: op.field_value(p, t), 0.0, T, limit=400, epsabs=1e-14)[0]
    assert abs(q - _sin2_pulse_area(p.E0, w, T)) < 1e-9 * abs(q)
    assert op.field_value(p, -0.5) == 0.0 and op.field_value(p, T + 0.5) == 0.0
    assert abs(op.field_value(p, 0.0)) < 1e-15 and abs(op.field_value(p, T)) < 1e-12 * p.E0


def observables_normalisation_errors():
    """Largest deviation of the oracle's (P_x, J_x, occ) from the single-k-point expectation
    values Tr(rho d), Tr(rho v), rho_c1c1 (scalar loops) for states that are the same at
    every k-point: the four-band model with one k-point's dipole, velocity and state copied
    to all 16 k-points, and the one-k-point two-band model.  Observables per unit cell
    (the 1/Nk reading of the k-sum) do not change when a k-point is repeated."""
    import copy
    rng = np.random.default_rng(8)
    errs = []
    for p, k0 in ((wl.small_model(4, 2), 5), (wl.small_model(1, 1), 0)):
        m = om.Model(p)
        Nb = m.Nb
        mt = copy.copy(m)
        mt.dx = np.broadcast_to(m.dx[k0], m.dx.shape).copy()
        mt.vx = np.broadcast_to(m.vx[k0], m.vx.shape).copy()
        X0 = rng.standard_normal((Nb, Nb)) + 1j * rng.standard_normal((Nb, Nb))
        X0 = 0.01 * (X0 + X0.conj().T)
        X = np.broadcast_to(X0, (m.Nk, Nb, Nb)).reshape(-1).copy()
        rho = np.diag(m.occ) + X0
        want = [0.0, 0.0, rho[m.c1, m.c1].real]
        for n in range(Nb):
            for mm in range(Nb):
                want[0] += (rho[n, mm] * m.dx[k0][mm, n]).real
                want[1] += (rho[n, mm] * m.vx[k0][mm, n]).real
        errs.append(np.abs(op.observables(mt, X) - np.array(want)).max())
    # physical case: a fraction f of each k-point's valence population moved to c1 gives
    # occupation f per unit cell on the real (k-dependent) model
    m = om.Model(wl.small_model(4, 2))
    f = 0.125
    X = np.zeros((m.Nk, m.Nb, m.Nb), complex)
    X[:, 0, 0], X[:, m.c1, m.c1] = -f, f
    errs.append(abs(op.observables(m, X.reshape(-1))[2] - f))
    return max(errs)


def test_observables_are_per_k_point_expectation_values():
    """P, J and occupation are per-unit-cell expectation values (the reading of the
    paper's unnormalised k-sums as (1/Nk) sum_k): a k-uniform state gives the one-k-point
    values; 1/N, 1/(Nk Nb) or a plain sum would scale them by Nb^-2, Nb^-1 or Nk."""
    assert observables_normalisation_errors() < 1e-15


def test_stationary_without_field(m4):
    K = ok.dense_kernel(m4)
    s = np.zeros(2 * 20 + 1)
    obs, x = op.rk4(m4, lambda v: K @ v, s, 0.2, 20)
    assert np.all(x == 0)
    assert np.all(obs[:, 0] == 0) and np.all(obs[:, 2] == 0)


def test_trace_and_hermiticity_conserved(m4):
    K = ok.dense_kernel(m4)
    pulse = wl.Pulse(E0=5e-3, omega=0.1, t0=10.0, sigma=5.0)
    T = 100
    _, x = op.rk4(m4, lambda v: K @ v, op.half_step_samples(pulse, 0.2, T), 0.2, T)
    X = x.reshape(m4.Nk, 4, 4)
    assert np.abs(np.trace(X, axis1=1, axis2=2)).max() < 1e-15
    assert np.abs(X - np.conj(np.swapaxes(X, 1, 2))).max() < 1e-15
    assert np.abs(X).max() > 1e-5


def test_gauge_invariance_of_observables(m4):
    """Random per-k band phases change K, d, v and rho, but not P, J, occupation."""
    rng = np.random.default_rng(2)
    m4b = m4.rephased(rng.uniform(0, 2 * np.pi, (m4.Nk, m4.Nb)))
    pulse = wl.Pulse(E0=5e-3, omega=0.1, t0=10.0, sigma=5.0)
    T = 60
    s = op.half_step_samples(pulse, 0.2, T)
    K1, K2 = ok.dense_kernel(m4), ok.dense_kernel(m4b)
    o1, _ = op.rk4(m4, lambda v: K1 @ v, s, 0.2, T)
    o2, _ = op.rk4(m4b, lambda v: K2 @ v, s, 0.2, T)
    assert np.abs(o1[:, 0]).max() > 1e-5
    np.testing.assert_allclose(o1, o2, atol=1e-15)


def test_lowrank_full_rank_propagation_equals_full(m2):
    K = ok.dense_kernel(m2)
    d, Koff = ok.split_diag_off(K)
    U, S, V = olr.truncated_svd(Koff, m2.N)
    pulse = wl.Pulse(E0=5e-3, omega=0.1, t0=10.0, sigma=5.0)
    T = 80
    s = op.half_step_samples(pulse, 0.2, T)
    o1, _ = op.rk4(m2, lambda v: K @ v, s, 0.2, T)
    o2, _ = op.rk4(m2, lambda v: olr.apply_lowrank(d, U, S, V, v), s, 0.2, T)
    assert op.rel_l2(o2[:, 0], o1[:, 0]) < 1e-12


def test_truncation_error_shrinks_with_rank():
    """Paper trend (Fig. abs_linear): P(t) error vs the full kernel falls as rank grows."""
    mdl = om.Model(wl.small_model(8, 1))
    K = ok.dense_kernel(mdl)
    d, Koff = ok.split_diag_off(K)
    pulse = wl.Pulse(E0=1e-3, omega=0.1, t0=40.0, sigma=12.0)
    T = 300
    s = op.half_step_samples(pulse, 0.2, T)
    ref, _ = op.rk4(mdl, lambda v: K @ v, s, 0.2, T)
    errs = []
    for r in (2, 13, 51, 128):
        U, S, V = olr.truncated_svd(Koff, r)
        o, _ = op.rk4(mdl, lambda v: olr.apply_lowrank(d, U, S, V, v), s, 0.2, T)
        errs.append(op.rel_l2(o[:, 0], ref[:, 0]))
    assert all(a > b for a, b in zip(errs, errs[1:])), errs


def test_linear_response_scaling(m2):
    """Weak field: P(t) is linear in E0 to O(E0^2) (linear-response limit of Eq. tdagw)."""
    K = ok.dense_kernel(m2)
    T = 150
    outs = []
    for E0 in (1e-5, 2e-5):
        s = op.half_step_samples(wl.Pulse(E0=E0, omega=0.1, t0=10.0, sigma=5.0), 0.2, T)
        outs.append(op.rk4(m2, lambda v: K @ v, s, 0.2, T)[0][:, 0])
    assert op.rel_l2(outs[1], 2 * outs[0]) < 1e-4
