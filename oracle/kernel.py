"""Electron-hole kernel K of the model, its diagonal/off-diagonal split, and K.x (FP64).

Test infrastructure only (see the package header).

Direct term (Eq. bse-direct-def) for the lattice model: the plane-wave matrix elements
M_{nn'}(k, q, G) are replaced by the Bloch overlaps <u_n(k)|u_n'(k')> (G = 0 only), and
W_{GG'}(q) by a 2D Rytova-Keldysh interaction, giving

  K_{(k n m),(k' n' m')} = - W(k - k') (U_k^+ U_k')_{n n'} (U_k'^+ U_k)_{m' m}

with the pair index i = (k Nb + n) Nb + m (row) and the density matrix rho_{n m k}
flattened the same way, so that dSigma = K . drho is Eq. sigma-from-k.

Readings (paper silent or garbled):
  * W(q) = 2 pi / (A |q| (1 + r0 |q|)) with A = Nk a^2, the Born-von Karman supercell
    area (the usual 1/(Nk Omega) normalisation of a k-sum).
  * q = k - k' is taken as the minimum image on the periodic grid.
  * q = 0 (Appendix B: "replace W(q=0) with an average over a small region of the
    Brillouin zone"): the average of W over the k-grid's own mini-cell, the square
    |qx|, |qy| <= h with h = pi / (L a).
  * Eq. sigma-from-k is applied to drho = rho - rho0 (dSigma = Sigma[G] - Sigma[G0]).
  * K^diag (Sec. "SVD analysis", "n1,n2,k = n3,n4,k'") is the strict matrix diagonal;
    split_kblocks gives the other reading, the k = k' blocks of Nb^2 x Nb^2.

Exchange term (Eq. bse-exchange-def at Q = 0), optional (ModelParams.exchange = lambda_x,
0 by default):

  K^x_{(k n m),(k' n' m')} = lambda_x sum_G v(G) M_nm(k, G) conj(M_n'm'(k', G)),
  M_nm(k, G) = sum_o conj(U_k[o, n]) U_k[o, m] exp(i G . tau_o),  v(G) = 2 pi / (A |G|).

Readings for the lattice model (no plane-wave basis): orbitals are points, orbital o of
each copy at tau_o = (o mod 2) (a/2, a/2); G runs over the first two shells of reciprocal
vectors (2 pi / a)(i, j), |i|, |j| <= 1, (i, j) != 0 (the G = 0 term, divergent at Q = 0,
is left out as in the paper's TDA absorption kernels).
"""
from __future__ import annotations

import numpy as np


def coulomb_W(qabs: np.ndarray, A: float, r0: float) -> np.ndarray:
    """2D Rytova-Keldysh interaction 2 pi / (A |q| (1 + r0 |q|)) for |q| > 0 (the screened
    W of Eq. bse-direct-def for the lattice model; Appendix B)."""
    return 2.0 * np.pi / (A * qabs * (1.0 + r0 * qabs))


def cell_average_W0(h: float, A: float, r0: float, npts: int = 64) -> float:
    """W(q = 0) as the average over a small region (Appendix B): the mean of W(q) over the
    square |qx|,|qy| <= h.

    In polar coordinates the square is 8 triangles 0 <= theta <= pi/4,
    0 <= |q| <= h / cos(theta); the radial integral of |q| W(q) is closed-form,
        int_0^R dq 2 pi / (A (1 + r0 q)) = (2 pi / (A r0)) ln(1 + r0 R),
    leaving one smooth angular integral done by Gauss-Legendre.
    """
    x, w = np.polynomial.legendre.leggauss(npts)
    theta = 0.25 * np.pi * 0.5 * (x + 1.0)
    wt = 0.25 * np.pi * 0.5 * w
    ang = np.sum(wt * np.log1p(r0 * h / np.cos(theta)))
    return 8.0 * (2.0 * np.pi / (A * r0)) * ang / (4.0 * h * h)


def min_image(d: np.ndarray, L: int) -> np.ndarray:
    """Integer offset wrapped into [-L/2, L/2) (q = k - k' on the periodic grid of Eq.
    bse-direct-def)."""
    return (d + L // 2) % L - L // 2


def W_of_offsets(di: np.ndarray, dj: np.ndarray, p) -> np.ndarray:
    """W of Eq. bse-direct-def on integer grid offsets (already minimum-image); the Appendix B
    average W0 at the origin."""
    L, a = p.L, p.a
    A = p.Nk * a * a
    qx = di * (2.0 * np.pi / (L * a))
    qy = dj * (2.0 * np.pi / (L * a))
    q = np.hypot(qx, qy)
    out = np.empty_like(q)
    nz = q > 0
    out[nz] = coulomb_W(q[nz], A, p.r0)
    out[~nz] = cell_average_W0(np.pi / (L * a), A, p.r0)
    return out


def W_matrix(p) -> np.ndarray:
    """W(k - k') of Eq. bse-direct-def for all pairs of grid points; (Nk, Nk)."""
    L = p.L
    ii, jj = np.divmod(np.arange(p.Nk), L)
    di = min_image(ii[:, None] - ii[None, :], L)
    dj = min_image(jj[:, None] - jj[None, :], L)
    return W_of_offsets(di, dj, p)


def exchange_vectors(model):
    """(M, v): M (Nk, nG, Nb, Nb) = M_nm(k, G) and v (nG,) = lambda_x v(G) for the eight
    reciprocal vectors of the exchange term of Eq. bse-exchange-def (see the module header)."""
    p = model.p
    A = p.Nk * p.a * p.a
    Gs = [(i, j) for i in (-1, 0, 1) for j in (-1, 0, 1) if (i, j) != (0, 0)]
    no = model.U.shape[1]
    tau = np.array([[(o % 2) * p.a / 2, (o % 2) * p.a / 2] for o in range(no)])
    M = np.empty((model.Nk, len(Gs), model.Nb, model.Nb), complex)
    v = np.empty(len(Gs))
    for g, (i, j) in enumerate(Gs):
        G = 2 * np.pi / p.a * np.array([i, j], float)
        ph = np.exp(1j * tau @ G)                                    # (no,)
        M[:, g] = np.einsum("kon,o,kom->knm", model.U.conj(), ph, model.U)
        v[g] = p.exchange * 2 * np.pi / (A * np.linalg.norm(G))
    return M, v


def exchange_kernel(model) -> np.ndarray:
    """The dense exchange term K^x of Eq. bse-exchange-def (N x N), zero when lambda_x = 0."""
    M, v = exchange_vectors(model)
    Mf = M.reshape(model.Nk, len(v), -1).transpose(1, 0, 2).reshape(len(v), -1)   # (nG, N)
    return np.einsum("g,gi,gj->ij", v, Mf, Mf.conj())


def dense_kernel(model) -> np.ndarray:
    """The full N x N kernel of Eq. sigma-from-k (complex128), straight from the entry
    formula of Eq. bse-direct-def (plus Eq. bse-exchange-def when lambda_x > 0)."""
    p, Nk, Nb = model.p, model.Nk, model.Nb
    W = W_matrix(p)
    U = model.U
    O = np.einsum("kin,qip->kqnp", U.conj(), U)          # O[k,k',n,n'] = (U_k^+ U_k')_{nn'}
    # (U_k'^+ U_k)_{m' m} = conj(O[k,k',m,m'])
    K = -W[:, :, None, None, None, None] * O[:, :, :, None, :, None] * \
        np.conj(O)[:, :, None, :, None, :]               # [k,k',n,m,n',m']
    K = np.transpose(K, (0, 2, 3, 1, 4, 5)).reshape(Nk * Nb * Nb, Nk * Nb * Nb)
    if getattr(p, "exchange", 0.0):
        K = K + exchange_kernel(model)
    return np.ascontiguousarray(K)


def kernel_entry(model, row: int, col: int) -> complex:
    """One entry K[row, col] by the formula of Eq. bse-direct-def (and Eq.
    bse-exchange-def) as a scalar loop, for sampled checks."""
    p, Nb = model.p, model.Nb
    k, rem = divmod(row, Nb * Nb)
    n, m = divmod(rem, Nb)
    kp, rem = divmod(col, Nb * Nb)
    n2, m2 = divmod(rem, Nb)
    L = p.L
    di = min_image(np.array([k // L - kp // L]), L)
    dj = min_image(np.array([k % L - kp % L]), L)
    W = W_of_offsets(di, dj, p)[0]
    Uk, Ukp = model.U[k], model.U[kp]
    o1 = np.vdot(Uk[:, n], Ukp[:, n2])
    o2 = np.vdot(Ukp[:, m2], Uk[:, m])
    val = complex(-W * o1 * o2)
    if getattr(p, "exchange", 0.0):
        M, v = exchange_vectors(model)
        for g in range(len(v)):
            val += v[g] * M[k, g, n, m] * np.conj(M[kp, g, n2, m2])
    return val


def kernel_row(model, row: int) -> np.ndarray:
    """Row `row` of K (Eq. bse-direct-def, and Eq. bse-exchange-def), length N, vectorised
    over columns; for sampled-row checks."""
    p, Nb, Nk = model.p, model.Nb, model.Nk
    k, rem = divmod(row, Nb * Nb)
    n, m = divmod(rem, Nb)
    L = p.L
    kp = np.arange(Nk)
    W = W_of_offsets(min_image(k // L - kp // L, L), min_image(k % L - kp % L, L), p)
    o1 = np.einsum("i,qip->qp", model.U[k, :, n].conj(), model.U)        # (Nk, n')
    o2 = np.einsum("qip,i->qp", model.U.conj(), model.U[k, :, m])        # (Nk, m')
    row_ = (-W[:, None, None] * o1[:, :, None] * o2[:, None, :]).reshape(-1)
    if getattr(p, "exchange", 0.0):
        M, v = exchange_vectors(model)
        row_ = row_ + np.einsum("g,g,qgab->qab", v, M[k, :, n, m], M.conj()).reshape(-1)
    return row_


def kernel_diag(model) -> np.ndarray:
    """diag(K), the strict-diagonal K^diag of Eq. svd_diag_offdiag, of the direct kernel:
    -W0 (U_k^+U_k)_{nn} (U_k^+U_k)_{mm}; length N."""
    p = model.p
    W0 = cell_average_W0(np.pi / (p.L * p.a), p.Nk * p.a * p.a, p.r0)
    g = np.einsum("kin,kin->kn", model.U.conj(), model.U).real
    d = (-W0 * g[:, :, None] * g[:, None, :]).reshape(-1).astype(np.complex128)
    if getattr(p, "exchange", 0.0):
        M, v = exchange_vectors(model)
        d = d + np.einsum("g,kgab->kab", v, np.abs(M) ** 2).reshape(-1)
    return d


def split_kblocks(K: np.ndarray, Nb: int):
    """The other reading of K^diag in Sec. "SVD analysis of electron-hole kernel": the
    k = k' blocks.  Returns (B, Koff) with B
    (Nk, P, P) the blocks K[k P + p, k P + q] (P = Nb^2) and Koff = K without them."""
    P = Nb * Nb
    Nk = K.shape[0] // P
    B = np.stack([K[k * P:(k + 1) * P, k * P:(k + 1) * P] for k in range(Nk)])
    Koff = K.copy()
    for k in range(Nk):
        Koff[k * P:(k + 1) * P, k * P:(k + 1) * P] = 0.0
    return B, Koff


def split_diag_off(K: np.ndarray):
    """K = K^diag + K^off with K^diag the strict matrix diagonal (Eq. svd_diag_offdiag)."""
    d = np.diag(K).copy()
    Koff = K.copy()
    np.fill_diagonal(Koff, 0.0)
    return d, Koff


def apply_dense(K: np.ndarray, x: np.ndarray) -> np.ndarray:
    """dSigma = K . x (Eq. sigma-from-k), one matrix-vector product."""
    return K @ x


def fft_applier(model):
    """K . x of Eq. sigma-from-k through the convolution structure of Eq. bse-direct-def (an
    identity, not a model).

    Summing the entry formula over n', m':
        (K x)_k = - U_k^+ [ sum_k' W(k - k') U_k' X_k' U_k'^+ ] U_k ,
    a circular 2D convolution over the periodic grid done with FFTs.  Costs
    O(N log Nk) instead of O(N^2); exact to rounding for any x.  Returns x -> K x.
    """
    p, L, Nb = model.p, model.L, model.Nb
    U = model.U
    no = U.shape[1]
    Uh = np.conj(np.swapaxes(U, 1, 2))
    di, dj = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    What = np.fft.fft2(W_of_offsets(min_image(di, L), min_image(dj, L), p))[:, :, None, None]

    exch = bool(getattr(p, "exchange", 0.0))
    if exch:
        M, v = exchange_vectors(model)
        Mf = M.reshape(model.Nk, len(v), -1).transpose(1, 0, 2).reshape(len(v), -1)   # (nG, N)

    def apply(x: np.ndarray) -> np.ndarray:
        X = x.reshape(model.Nk, Nb, Nb)
        Y = (U @ X @ Uh).reshape(L, L, no, no)                       # orbital basis
        Z = np.fft.ifft2(What * np.fft.fft2(Y, axes=(0, 1)), axes=(0, 1))
        out = (-(Uh @ Z.reshape(model.Nk, no, no) @ U)).reshape(-1)
        if exch:   # the exchange term through its rank-nG form
            out = out + Mf.T @ (v * (Mf.conj() @ x))
        return out

    return apply


def apply_fft(model, x: np.ndarray) -> np.ndarray:
    """One K . x of Eq. sigma-from-k by the FFT form (see fft_applier)."""
    return fft_applier(model)(x)
