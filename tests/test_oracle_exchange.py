"""Pins of the exchange term (Eq. bse-exchange-def for the lattice model) and of the k-block
reading of K^diag.  No GPU."""
import dataclasses

import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import kernel as ok
from oracle import lowrank as olr
from oracle import model as om


def _model(L, nc, lx):
    return om.Model(dataclasses.replace(wl.small_model(L, nc), exchange=lx))


@pytest.fixture(scope="module")
def mx():
    return _model(5, 2, 1.0)


def test_exchange_entries_by_scalar_loops(mx):
    """Entries of K^x by explicit loops over the eight reciprocal vectors and the orbitals,
    with the phases exp(i G . tau) from cos/sin."""
    p, U = mx.p, mx.U
    Kx = ok.exchange_kernel(mx)
    A = p.Nk * p.a * p.a
    rng = np.random.default_rng(1)
    Nb = mx.Nb
    for _ in range(20):
        r, c = rng.integers(0, mx.N, 2)
        k, rem = divmod(int(r), Nb * Nb)
        n, m = divmod(rem, Nb)
        kp, rem = divmod(int(c), Nb * Nb)
        n2, m2 = divmod(rem, Nb)
        val = 0j
        for i in (-1, 0, 1):
            for j in (-1, 0, 1):
                if i == 0 and j == 0:
                    continue
                gx, gy = 2 * np.pi * i / p.a, 2 * np.pi * j / p.a
                v = 2 * np.pi / (A * np.hypot(gx, gy))
                Mk = Mkp = 0j
                for o in range(U.shape[1]):
                    t = (o % 2) * p.a / 2
                    ph = complex(np.cos(gx * t + gy * t), np.sin(gx * t + gy * t))
                    Mk += np.conj(U[k, o, n]) * U[k, o, m] * ph
                    Mkp += np.conj(U[kp, o, n2]) * U[kp, o, m2] * ph
                val += v * Mk * np.conj(Mkp)
        assert abs(Kx[r, c] - val) < 1e-15


def test_exchange_hermitian_low_rank_and_scaled(mx):
    """K^x is Hermitian and of rank 2: the phases exp(i G . tau) = (-1)^((i+j)(o mod 2)) give
    one matrix element pattern per shell; it scales linearly with lambda_x."""
    Kx = ok.exchange_kernel(mx)
    np.testing.assert_allclose(Kx, Kx.conj().T, atol=1e-16)
    ev = np.abs(scipy.linalg.eigvalsh(Kx))
    assert (ev > 1e-12 * ev.max()).sum() == 2
    np.testing.assert_allclose(ok.exchange_kernel(_model(5, 2, 3.0)), 3 * Kx, rtol=1e-13, atol=1e-18)
    assert np.abs(ok.exchange_kernel(_model(5, 2, 0.0))).max() == 0


def test_kernel_with_exchange_equals_fft_form_and_is_gauge_covariant(mx):
    K = ok.dense_kernel(mx)
    x = wl.random_state(mx.N, 4)
    np.testing.assert_allclose(ok.apply_fft(mx, x), K @ x, atol=1e-13 * np.abs(K @ x).max())
    ph = np.random.default_rng(2).uniform(0, 2 * np.pi, (mx.Nk, mx.Nb))
    K2 = ok.dense_kernel(mx.rephased(ph))
    e = np.exp(1j * ph)
    pair = (e.conj()[:, :, None] * e[:, None, :]).reshape(-1)
    np.testing.assert_allclose(K2, pair[:, None] * K * pair.conj()[None, :], atol=1e-15)
    rows = [0, 7, mx.N - 1]
    for r in rows:
        np.testing.assert_allclose(ok.kernel_row(mx, r), K[r], atol=1e-16)
        assert abs(ok.kernel_entry(mx, r, (r * 13) % mx.N) - K[r, (r * 13) % mx.N]) < 1e-16
    np.testing.assert_allclose(ok.kernel_diag(mx), np.diag(K), atol=1e-16)


def test_direct_kernel_k_blocks_are_minus_W0_identity():
    """Without exchange the k = k' block of the direct kernel is -W0 (U_k^+ U_k) x (U_k^+ U_k)
    = -W0 I: the k-block reading of K^diag coincides with the strict diagonal."""
    m = _model(6, 2, 0.0)
    K = ok.dense_kernel(m)
    B, Koff = ok.split_kblocks(K, m.Nb)
    W0 = ok.cell_average_W0(np.pi / (m.p.L * m.p.a), m.p.Nk * m.p.a ** 2, m.p.r0)
    np.testing.assert_allclose(B, np.broadcast_to(-W0 * np.eye(m.Nb ** 2), B.shape), atol=1e-16)
    d, Ks = ok.split_diag_off(K)
    np.testing.assert_allclose(Koff, Ks, atol=1e-16)


def test_k_block_split_with_exchange(mx):
    """With exchange the blocks are Hermitian and not diagonal; K = blocks + Koff; Koff has
    zero k = k' blocks; the low-rank apply with blocks at full rank reproduces K."""
    K = ok.dense_kernel(mx)
    B, Koff = ok.split_kblocks(K, mx.Nb)
    P = mx.Nb ** 2
    np.testing.assert_allclose(B, np.conj(np.swapaxes(B, 1, 2)), atol=1e-16)
    off = B - np.einsum("kpp->kp", B)[:, :, None] * np.eye(P)
    assert np.abs(off).max() > 1e-4 * np.abs(B).max()
    rebuilt = Koff.copy()
    for k in range(mx.Nk):
        assert np.abs(Koff[k * P:(k + 1) * P, k * P:(k + 1) * P]).max() == 0
        rebuilt[k * P:(k + 1) * P, k * P:(k + 1) * P] = B[k]
    np.testing.assert_array_equal(rebuilt, K)
    U, S, V = olr.truncated_svd(Koff, mx.N)
    x = wl.random_state(mx.N, 5)
    np.testing.assert_allclose(olr.apply_lowrank_kblocks(B, U, S, V, x), K @ x, atol=1e-12 * np.abs(K @ x).max())


def test_strict_split_compresses_better_with_exchange():
    """The rank-2 exchange term stays low rank only as a whole: cutting its k = k' blocks out
    (the k-block reading) leaves a remainder of higher rank, so at equal rank the strict
    diagonal split truncates with the smaller error on this model."""
    m = _model(8, 2, 1.0)
    K = ok.dense_kernel(m)
    _, Koff_b = ok.split_kblocks(K, m.Nb)
    _, Koff_s = ok.split_diag_off(K)
    sb = np.sort(np.abs(scipy.linalg.eigvalsh(Koff_b)))[::-1]
    ss = np.sort(np.abs(scipy.linalg.eigvalsh(Koff_s)))[::-1]
    for r in (20, 51, 102):
        assert np.sum(ss[r:] ** 2) < np.sum(sb[r:] ** 2)


def test_kblock_adjoint_operator_dot_product(mx):
    """<u, K~ v> = <K~^H u, v> for the k-block low-rank form, with K~^H applying the
    conjugate-transposed blocks and V S U^H."""
    K = ok.dense_kernel(mx)
    B, Koff = ok.split_kblocks(K, mx.Nb)
    U, S, V = olr.truncated_svd(Koff, 11)
    BH = np.conj(np.swapaxes(B, 1, 2))
    rng = np.random.default_rng(8)
    u = rng.standard_normal(mx.N) + 1j * rng.standard_normal(mx.N)
    v = rng.standard_normal(mx.N) + 1j * rng.standard_normal(mx.N)
    Kv = olr.apply_lowrank_kblocks(B, U, S, V, v)
    KHu = np.einsum("kpq,kq->kp", BH, u.reshape(mx.Nk, -1)).reshape(-1) + V @ (S * (U.conj().T @ u))
    assert abs(np.vdot(u, Kv) - np.vdot(KHu, v)) < 1e-12 * np.abs(np.vdot(u, Kv))
