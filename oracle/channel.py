"""Channel-wise truncated SVD of the kernel and its apply (FP64).

Test infrastructure only (see the package header).

Sec. "SVD analysis of electron-hole kernel", Eq. svd-channel-wise: a channel
ch = (n1 n2) -> (n3 n4) is the Nk x Nk block

    K^ch[k, k'] = K_{(k n1 n2), (k' n3 n4)},

and each channel is compressed on its own by a truncated SVD over (k, k'),
K^ch ~ U^ch diag(S^ch) (V^ch)^H, keeping its z' largest singular triplets.

Readings (paper silent or garbled):
  * As for Eq. svd_diag_offdiag, the right factor (V~^ch)^T of a complex channel is the
    conjugate transpose (V^ch)^H.
  * Diagonal channels (n1 n2 = n3 n4, close to full rank) are kept exact and the
    off-diagonal channels are truncated to one common rank z': the kernels
    "K_0^diag-ch + z' K_0^off-ch" of Sec. "SVD compression for GW-BSE within TDA"
    (z' = 0 is "K_0^diag-ch only").
  * Pair index p = n1 Nb + n2, the flattening of the density matrix (k Nb + n) Nb + m, so
    row (k, p) of K is row k Nb^2 + p.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from oracle import kernel as ok


def channel_block(K: np.ndarray, Nb: int, p: int, q: int) -> np.ndarray:
    """K^ch of Eq. svd-channel-wise for ch = p -> q: rows k Nb^2 + p, columns k' Nb^2 + q
    (Nk x Nk copy)."""
    P = Nb * Nb
    return K[p::P, q::P].copy()


def channel_block_from_model(model, p: int, q: int, W: np.ndarray | None = None) -> np.ndarray:
    """K^pq (Eq. svd-channel-wise) straight from the entry formula of Eq. bse-direct-def,
    without the dense N x N kernel (for
    large grids): with p = (n1, n2), q = (n3, n4) and O_ab[k, k'] = (U_k^+ U_k')_{ab},
        K^pq[k, k'] = -W(k - k') O_{n1 n3}[k, k'] conj(O_{n2 n4}[k, k']),
    since (U_k'^+ U_k)_{n4 n2} = conj((U_k^+ U_k')_{n2 n4})."""
    Nb = model.Nb
    n1, n2 = divmod(p, Nb)
    n3, n4 = divmod(q, Nb)
    U = model.U
    o13 = U[:, :, n1].conj() @ U[:, :, n3].T
    o24 = U[:, :, n2].conj() @ U[:, :, n4].T
    if W is None:
        W = ok.W_matrix(model.p)
    return -W * o13 * o24.conj()


def channel_svd(K: np.ndarray, Nb: int, rank: int):
    """Eq. svd-channel-wise with exact LAPACK SVDs (gesdd) of every off-diagonal channel.

    Returns (D, U, S, V): D (P, Nk, Nk) the dense diagonal channels K^{pp}; U, V
    (P, P, Nk, rank) and S (P, P, rank) the top-`rank` singular triplets of K^{pq} for
    p != q (zero for p == q).  P = Nb^2; `rank` <= Nk.
    """
    P = Nb * Nb
    Nk = K.shape[0] // P
    assert 0 <= rank <= Nk
    D = np.zeros((P, Nk, Nk), complex)
    U = np.zeros((P, P, Nk, rank), complex)
    V = np.zeros((P, P, Nk, rank), complex)
    S = np.zeros((P, P, rank))
    for p in range(P):
        D[p] = channel_block(K, Nb, p, p)
        for q in range(P):
            if q == p or rank == 0:
                continue
            u, s, vh = scipy.linalg.svd(channel_block(K, Nb, p, q), full_matrices=False,
                                        lapack_driver="gesdd")
            U[p, q] = u[:, :rank]
            S[p, q] = s[:rank]
            V[p, q] = vh[:rank].conj().T
    return D, U, S, V


def channel_svd_from_model(model, rank: int):
    """Eq. svd-channel-wise as channel_svd, without the dense N x N kernel (large grids):
    every channel from the
    kernel's entry formula (channel_block_from_model); vanishing channels keep zero factors."""
    Nb, Nk = model.Nb, model.Nk
    P = Nb * Nb
    D = np.zeros((P, Nk, Nk), complex)
    U = np.zeros((P, P, Nk, rank), complex)
    V = np.zeros((P, P, Nk, rank), complex)
    S = np.zeros((P, P, rank))
    W = ok.W_matrix(model.p)
    for p in range(P):
        for q in range(P):
            blk = channel_block_from_model(model, p, q, W)
            if p == q:
                D[p] = blk
            elif rank > 0 and np.abs(blk).max() > 0:
                u, s, vh = scipy.linalg.svd(blk, full_matrices=False, lapack_driver="gesdd")
                U[p, q] = u[:, :rank]
                S[p, q] = s[:rank]
                V[p, q] = vh[:rank].conj().T
    return D, U, S, V


def apply_channel(D, U, S, V, x: np.ndarray) -> np.ndarray:
    """dSigma = K~ x (Eq. sigma-from-k) for the channel-wise kernel of Eq. svd-channel-wise:

        dSigma[(k, p)] = sum_k' D^p[k, k'] x[(k', p)]
                       + sum_{q != p} U^{pq} diag(S^{pq}) (V^{pq})^H x_q,

    with x_q[k'] = x[(k', q)]; the diagonal channels (p == q) take only D."""
    P = D.shape[0]
    Nk = D.shape[1]
    xs = x.reshape(Nk, P)
    out = np.zeros((Nk, P), complex)
    for p in range(P):
        out[:, p] = D[p] @ xs[:, p]
        for q in range(P):
            if q == p:
                continue
            out[:, p] += U[p, q] @ (S[p, q] * (V[p, q].conj().T @ xs[:, q]))
    return out.reshape(-1)


def assemble(D, U, S, V) -> np.ndarray:
    """The dense N x N matrix of the channel-wise kernel (Eq. svd-channel-wise), channel by
    channel."""
    P, Nk = D.shape[0], D.shape[1]
    K = np.zeros((P * Nk, P * Nk), complex)
    for p in range(P):
        for q in range(P):
            blk = D[p] if p == q else (U[p, q] * S[p, q]) @ V[p, q].conj().T
            K[p::P, q::P] = blk
    return K


def channel_singular_values(K: np.ndarray, Nb: int) -> np.ndarray:
    """Singular values of every channel, (P, P, Nk), descending (Fig. svd_analysis(b))."""
    P = Nb * Nb
    Nk = K.shape[0] // P
    out = np.zeros((P, P, Nk))
    for p in range(P):
        for q in range(P):
            out[p, q] = scipy.linalg.svdvals(channel_block(K, Nb, p, q))
    return out
