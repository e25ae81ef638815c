"""Tight-binding model: k-grid, bands, eigenvectors, dipoles and velocity (FP64).

Test infrastructure only (see the package header).

The paper's bands come from DFT + G0W0 (Appendix A); H^QP is diagonal in the band basis
(Eq. tdagw, second line: (eps_n - eps_m) rho_nm).  Here a two-band lattice model stands in:

  h(k) = Delta sz + t (sin(kx a) sx + sin(ky a) sy) + m (2 - cos(kx a) - cos(ky a)) sz

Readings (paper silent):
  * "sin kx" is sin(kx a): k carries units of 1/bohr, a in bohr.
  * Four bands = block-diag(h(k) + off_0 I, h(k) + off_1 I); bands are sorted by energy,
    the lower half is valence.
  * Gauge of each eigenvector: its largest-modulus orbital component is real and > 0.
  * Dipoles r (Appendix A.1, "locally smooth gauge equivalent to the parallel transport
    gauge"): k-local Berry connection A_nm = i <u_n(k)| d/dk u_m(k)> by central differences
    at k +- delta with delta = 1e-5 / a, each u_m(k +- delta) phase-aligned to u_m(k)
    (overlap real > 0), then Hermitised; the diagonal, zero in the parallel-transport
    gauge, is set to zero.  The intraband grad_k rho term is dropped: the
    paper's r is a fixed k-local matrix in C^{Nb^2 Nk x 3}.
  * Velocity (Sec. "SVD acceleration", J = Tr(rho v)): v_nm = <u_n| dh/dk |u_m>.
"""
from __future__ import annotations

import numpy as np

SX = np.array([[0, 1], [1, 0]], dtype=np.complex128)
SY = np.array([[0, -1j], [1j, 0]], dtype=np.complex128)
SZ = np.array([[1, 0], [0, -1]], dtype=np.complex128)


def kgrid(L: int, a: float) -> np.ndarray:
    """Gamma-centred unshifted L x L grid (the k-grids of Appendix A), k = (2 pi / (L a)) (i, j);
    index k = i*L + j."""
    i, j = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    k = np.stack([i.ravel(), j.ravel()], axis=1).astype(np.float64)
    return k * (2.0 * np.pi / (L * a))


def h_orbital(k: np.ndarray, p) -> np.ndarray:
    """Orbital-basis lattice Hamiltonian standing in for the quasiparticle bands H^QP of Eq.
    tdagw (Appendix A's are first-principles); shape (..., Norb, Norb), Norb = 2 nb_copies."""
    k = np.asarray(k, dtype=np.float64)
    kx, ky = k[..., 0] * p.a, k[..., 1] * p.a
    dx = p.t * np.sin(kx)
    dy = p.t * np.sin(ky)
    dz = p.Delta + p.m * (2.0 - np.cos(kx) - np.cos(ky))
    blk = (dx[..., None, None] * SX + dy[..., None, None] * SY + dz[..., None, None] * SZ)
    nc = p.nb_copies
    H = np.zeros(k.shape[:-1] + (2 * nc, 2 * nc), dtype=np.complex128)
    for c in range(nc):
        H[..., 2 * c:2 * c + 2, 2 * c:2 * c + 2] = blk + p.offsets[c] * np.eye(2)
    return H


def dh_dk(k: np.ndarray, p, axis: int) -> np.ndarray:
    """Analytic derivative dh/dk_axis of the stand-in bands of H^QP (Eq. tdagw), orbital
    basis, shape (..., Norb, Norb)."""
    k = np.asarray(k, dtype=np.float64)
    kx, ky = k[..., 0] * p.a, k[..., 1] * p.a
    ka = kx if axis == 0 else ky
    sig = SX if axis == 0 else SY
    blk = p.a * (p.t * np.cos(ka)[..., None, None] * sig + p.m * np.sin(ka)[..., None, None] * SZ)
    nc = p.nb_copies
    D = np.zeros(k.shape[:-1] + (2 * nc, 2 * nc), dtype=np.complex128)
    for c in range(nc):
        D[..., 2 * c:2 * c + 2, 2 * c:2 * c + 2] = blk
    return D


def fix_gauge(U: np.ndarray) -> np.ndarray:
    """Rephase each column so that its largest-modulus component is real and positive (a
    gauge choice; the observables of Eq. tdagw do not depend on it)."""
    U = np.array(U, dtype=np.complex128, copy=True)
    idx = np.argmax(np.abs(U), axis=-2)                       # (..., Nb)
    piv = np.take_along_axis(U, idx[..., None, :], axis=-2)   # (..., 1, Nb)
    return U * (np.abs(piv) / piv)


def eigensystem(k: np.ndarray, p):
    """Quasiparticle energies and states of the stand-in H^QP (Eq. tdagw): bands sorted
    ascending and gauge-fixed eigenvectors (columns), via LAPACK eigh."""
    eps, U = np.linalg.eigh(h_orbital(k, p))
    return eps, fix_gauge(U)


def _transported(Uk: np.ndarray, Ush: np.ndarray) -> np.ndarray:
    """Phase-align each column of Ush to the matching column of Uk (overlap real > 0)."""
    ov = np.einsum("...in,...in->...n", Uk.conj(), Ush)
    return Ush * (np.abs(ov) / ov)[..., None, :]


def berry_dipole(k: np.ndarray, p, axis: int, delta: float | None = None) -> np.ndarray:
    """The k-local position operator r of Eq. tdagw (length gauge; r in C^{Nb^2 Nk x 3},
    Appendix A.1) as the finite-difference Berry connection A_nm = i<u_n|du_m/dk>,
    Hermitised; (Nk, Nb, Nb)."""
    if delta is None:
        delta = 1e-5 / p.a
    e = np.zeros(2)
    e[axis] = delta
    _, U0 = eigensystem(k, p)
    _, Up = eigensystem(k + e, p)
    _, Um = eigensystem(k - e, p)
    Up = _transported(U0, Up)
    Um = _transported(U0, Um)
    dU = (Up - Um) / (2.0 * delta)
    A = 1j * np.einsum("...in,...im->...nm", U0.conj(), dU)
    A = 0.5 * (A + np.conj(np.swapaxes(A, -1, -2)))
    # parallel transport makes <u_m|du_m> vanish: the diagonal is zero by the gauge
    # condition, so rounding noise of the difference quotient is not kept
    idx = np.arange(A.shape[-1])
    A[..., idx, idx] = 0.0
    return A


def velocity(k: np.ndarray, p, axis: int) -> np.ndarray:
    """The velocity operator of the current J = Tr(rho v) (Sec. "SVD acceleration of
    TD-aGW"): v_nm = <u_n| dh/dk_axis |u_m> in the band basis; (Nk, Nb, Nb)."""
    _, U = eigensystem(k, p)
    return np.einsum("...in,...ij,...jm->...nm", U.conj(), dh_dk(k, p, axis), U)


class Model:
    """All k-local quantities of the model on its grid (FP64)."""

    def __init__(self, p):
        self.p = p
        self.L, self.Nb, self.Nk, self.N = p.L, p.Nb, p.Nk, p.N
        self.k = kgrid(p.L, p.a)
        self.eps, self.U = eigensystem(self.k, p)            # (Nk, Nb), (Nk, Norb, Nb)
        self.occ = np.zeros(self.Nb)
        self.occ[: self.Nb // 2] = 1.0                       # filled valence, empty conduction
        self.dx = berry_dipole(self.k, p, 0)
        self.dy = berry_dipole(self.k, p, 1)
        self.vx = velocity(self.k, p, 0)
        self.c1 = self.Nb // 2                               # first conduction band

    def rho0(self) -> np.ndarray:
        """Equilibrium density matrix: diag(occ) at every k; (Nk, Nb, Nb)."""
        return np.broadcast_to(np.diag(self.occ).astype(np.complex128),
                               (self.Nk, self.Nb, self.Nb)).copy()

    def rephased(self, phases: np.ndarray) -> "Model":
        """Same model in another band gauge: u_nk -> exp(i phi_nk) u_nk (for gauge tests).

        Dipoles and velocity transform covariantly, X_nm -> exp(-i phi_n) X_nm exp(i phi_m).
        """
        m = object.__new__(Model)
        m.__dict__.update(self.__dict__)
        ph = np.exp(1j * phases)                              # (Nk, Nb)
        m.U = self.U * ph[:, None, :]
        cov = ph.conj()[:, :, None] * ph[:, None, :]
        m.dx, m.dy, m.vx = self.dx * cov, self.dy * cov, self.vx * cov
        return m
