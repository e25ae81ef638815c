"""Truncated SVD of K^off and the low-rank apply (FP64).

Test infrastructure only (see the package header).

Eq. svd_diag_offdiag:  K ~ K^diag + U~ M~ V~^T with the z largest singular triplets of
K^off.  Reading: for a complex kernel the right factor is V^H (the paper's V~^T is the
conjugate transpose), i.e. K^off ~ U diag(S) V^H.  Eq. svd_acc applies it as
S~ (V~^H rho) with S~ = U~ M~, i.e. project first, then map back.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def truncated_svd(Koff: np.ndarray, rank: int):
    """Eq. svd_diag_offdiag: the top-`rank` singular triplets of K^off by LAPACK (gesdd):
    U (N,r), S (r,), V (N,r)."""
    U, S, Vh = scipy.linalg.svd(Koff, full_matrices=False, lapack_driver="gesdd")
    return U[:, :rank].copy(), S[:rank].copy(), Vh[:rank].conj().T.copy()


def singular_values(Koff: np.ndarray) -> np.ndarray:
    """Singular values of K^off, descending (the spectra of Fig. svd_analysis)."""
    return scipy.linalg.svdvals(Koff)


def apply_lowrank(diag: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray,
                  x: np.ndarray) -> np.ndarray:
    """dSigma = K^diag x + U (S * (V^H x)) (Eq. svd_acc)."""
    y = V.conj().T @ x
    return diag * x + U @ (S * y)


def apply_lowrank_kblocks(B: np.ndarray, U: np.ndarray, S: np.ndarray, V: np.ndarray,
                          x: np.ndarray) -> np.ndarray:
    """Eq. svd_acc with K^diag read as the k = k' blocks (Sec. "SVD analysis of
    electron-hole kernel"): dSigma = K^diag x + U (S * (V^H x)) with B (Nk, P, P):
    (K^diag x)[k P + p] = sum_q B[k, p, q] x[k P + q]."""
    Nk, P = B.shape[0], B.shape[1]
    y = V.conj().T @ x
    return np.einsum("kpq,kq->kp", B, x.reshape(Nk, P)).reshape(-1) + U @ (S * y)


def reconstruct(diag, U, S, V) -> np.ndarray:
    """The dense kernel of Eq. svd_diag_offdiag: diag(K) + U diag(S) V^H."""
    return np.diag(diag) + (U * S) @ V.conj().T


def r_squared(y: np.ndarray, yhat: np.ndarray) -> float:
    """R^2 = 1 - sum |y - yhat|^2 / sum |y - mean(y)|^2 (Sec. "SVD analysis"); for complex
    entries the squares are squared moduli and the mean is the complex mean."""
    y = np.asarray(y).ravel()
    yhat = np.asarray(yhat).ravel()
    return float(1.0 - np.sum(np.abs(y - yhat) ** 2) / np.sum(np.abs(y - y.mean()) ** 2))
