"""Pins of the channel-wise oracle (Eq. svd-channel-wise) against brute force, the
structure of the kernel and the Eckart-Young theorem.  No GPU.

A transposed channel (p and q swapped), a wrong pair index, a dropped diagonal channel or
a missing conjugation on V each fail one of these.
"""
import numpy as np
import pytest
import scipy.linalg

import workloads as wl
from oracle import channel as oc
from oracle import kernel as ok
from oracle import model as om
from oracle import propagate as op


@pytest.fixture(scope="module")
def k2():
    m = om.Model(wl.small_model(5, 1))
    return m, ok.dense_kernel(m)


@pytest.fixture(scope="module")
def k4():
    m = om.Model(wl.small_model(3, 2))
    return m, ok.dense_kernel(m)


def test_channel_block_indexing_by_integer_matrix():
    """Block p -> q of a matrix with entries row * N + col holds exactly the rows k P + p and
    columns k' P + q."""
    Nb, Nk = 2, 5
    P, N = Nb * Nb, Nb * Nb * Nk
    A = np.arange(N * N, dtype=float).reshape(N, N)
    for p in range(P):
        for q in range(P):
            blk = oc.channel_block(A, Nb, p, q)
            for k in range(Nk):
                for kp in range(Nk):
                    assert blk[k, kp] == (k * P + p) * N + kp * P + q


@pytest.mark.parametrize("name", ["k2", "k4"])
def test_channel_block_from_model_matches_dense_kernel(name, request):
    m, K = request.getfixturevalue(name)
    Nb = m.p.Nb
    for p in range(Nb * Nb):
        for q in range(Nb * Nb):
            np.testing.assert_allclose(oc.channel_block_from_model(m, p, q), oc.channel_block(K, Nb, p, q),
                                       atol=1e-15 * np.abs(K).max())


def test_channel_svd_from_model_matches_dense_route(k4):
    """The large-grid route (blocks from the formula, vanishing channels skipped) gives the
    same diagonal channels and the same truncated channels as the dense-kernel route."""
    m, K = k4
    r = 4
    D1, U1, S1, V1 = oc.channel_svd(K, m.Nb, r)
    D2, U2, S2, V2 = oc.channel_svd_from_model(m, r)
    np.testing.assert_allclose(D2, D1, atol=1e-15)
    np.testing.assert_allclose(S2, S1, atol=1e-14)
    for p in range(m.Nb ** 2):
        for q in range(m.Nb ** 2):
            if p != q:
                a = (U1[p, q] * S1[p, q]) @ V1[p, q].conj().T
                b = (U2[p, q] * S2[p, q]) @ V2[p, q].conj().T
                np.testing.assert_allclose(b, a, atol=1e-14)


def test_apply_channel_by_scalar_loops():
    """The channel apply against the sum written out element by element (random factors,
    tiny sizes), with the conjugate on V and the dense diagonal channels."""
    rng = np.random.default_rng(3)
    Nb, Nk, r = 2, 3, 2
    P = Nb * Nb
    cz = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)  # noqa: E731
    D, U, V, S = cz(P, Nk, Nk), cz(P, P, Nk, r), cz(P, P, Nk, r), rng.random((P, P, r))
    x = cz(P * Nk)
    got = oc.apply_channel(D, U, S, V, x)
    want = np.zeros(P * Nk, complex)
    for k in range(Nk):
        for p in range(P):
            acc = 0j
            for kp in range(Nk):
                acc += D[p, k, kp] * x[kp * P + p]
            for q in range(P):
                if q == p:
                    continue
                for j in range(r):
                    proj = 0j
                    for kp in range(Nk):
                        proj += np.conj(V[p, q, kp, j]) * x[kp * P + q]
                    acc += U[p, q, k, j] * S[p, q, j] * proj
            want[k * P + p] = acc
    np.testing.assert_allclose(got, want, rtol=1e-13, atol=1e-13)
    np.testing.assert_allclose(oc.assemble(D, U, S, V) @ x, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("name", ["k2", "k4"])
def test_full_rank_channels_reproduce_kernel(name, request):
    m, K = request.getfixturevalue(name)
    Nk = m.p.L ** 2
    D, U, S, V = oc.channel_svd(K, m.p.Nb, Nk)
    np.testing.assert_allclose(oc.assemble(D, U, S, V), K, atol=1e-13 * np.abs(K).max())
    x = np.random.default_rng(1).standard_normal(K.shape[0]) * (1 + 0.3j)
    np.testing.assert_allclose(oc.apply_channel(D, U, S, V, x), K @ x, atol=1e-12 * np.abs(K @ x).max())


def test_rank_zero_keeps_exactly_the_diagonal_channels(k2):
    """z' = 0 ("K_0^diag-ch only"): the kernel with every entry between different pairs
    removed, i.e. K masked by (i mod P == j mod P)."""
    m, K = k2
    P = m.p.Nb ** 2
    D, U, S, V = oc.channel_svd(K, m.p.Nb, 0)
    i = np.arange(K.shape[0])
    mask = (i[:, None] % P) == (i[None, :] % P)
    np.testing.assert_array_equal(oc.assemble(D, U, S, V), np.where(mask, K, 0))


@pytest.mark.parametrize("rank", [1, 4, 11])
def test_channel_eckart_young(k2, rank):
    """Each truncated channel misses the kernel by exactly the tail of its singular values."""
    m, K = k2
    Nb = m.p.Nb
    D, U, S, V = oc.channel_svd(K, Nb, rank)
    for p in range(Nb * Nb):
        for q in range(Nb * Nb):
            if p == q:
                continue
            blk = oc.channel_block(K, Nb, p, q)
            sv = scipy.linalg.svdvals(blk)
            err = np.linalg.norm(blk - (U[p, q] * S[p, q]) @ V[p, q].conj().T)
            assert abs(err - np.sqrt(np.sum(sv[rank:] ** 2))) < 1e-12 * sv[0]
            assert np.all(np.diff(S[p, q]) <= 0)


def test_hermitian_kernel_pairs_channels(k2):
    """K Hermitian => K^qp = (K^pq)^H, so both channels have the same singular values."""
    m, K = k2
    Nb = m.p.Nb
    sv = oc.channel_singular_values(K, Nb)
    for p in range(Nb * Nb):
        for q in range(Nb * Nb):
            np.testing.assert_allclose(oc.channel_block(K, Nb, q, p), oc.channel_block(K, Nb, p, q).conj().T)
            np.testing.assert_allclose(sv[p, q], sv[q, p], atol=1e-14 * sv.max())


def test_cross_copy_channels_vanish(k4):
    """Four bands from two decoupled copies: the overlaps between bands of different copies
    vanish, so channel (n1 n2) -> (n3 n4) is zero exactly when n1, n3 or n2, n4 belong to
    different copies.  The copy of each band is read off its orbital weights (orbitals
    0, 1: copy 0; 2, 3: copy 1), the same at every k."""
    m, K = k4
    Nb = m.p.Nb
    w1 = np.sum(np.abs(m.U[:, 2:, :]) ** 2, axis=1)        # (Nk, Nb) weight on copy 1
    copy = (w1[0] > 0.5).astype(int)
    assert np.all((w1 > 0.5) == copy[None, :]) and np.all((w1 < 1e-20) | (w1 > 1 - 1e-12))
    assert sorted(copy) == [0, 0, 1, 1]
    for p in range(Nb * Nb):
        n1, n2 = divmod(p, Nb)
        for q in range(Nb * Nb):
            n3, n4 = divmod(q, Nb)
            blk = oc.channel_block(K, Nb, p, q)
            same = copy[n1] == copy[n3] and copy[n2] == copy[n4]
            if same:
                assert np.abs(blk).max() > 1e-6
            else:
                assert np.abs(blk).max() < 1e-15


def test_diagonal_channels_need_more_rank_than_off_diagonal():
    """Sec. "SVD analysis": diagonal channels are close to full rank, off-diagonal ones are
    compressible.  On the two-band 12 x 12 model, the fraction of singular values needed for
    R^2 = 0.98 (the paper's criterion; by Eckart-Young the residual of the best rank-r
    approximation is the tail sum of squared singular values) is above 0.9 for every
    diagonal channel and below 0.4 for every off-diagonal one (paper, MoS2: 0.95 and 0.12
    on average)."""
    m = om.Model(wl.small_model(12, 1))
    K = ok.dense_kernel(m)
    Nb, Nk = m.p.Nb, m.p.L ** 2
    sv = oc.channel_singular_values(K, Nb)

    def ratio(p, q):
        blk = oc.channel_block(K, Nb, p, q)
        sst = np.sum(np.abs(blk - blk.mean()) ** 2)
        tail = np.concatenate([np.cumsum((sv[p, q] ** 2)[::-1])[::-1], [0.0]])
        return int(np.argmax(tail <= 0.02 * sst)) / Nk
    P = Nb * Nb
    assert min(ratio(p, p) for p in range(P)) > 0.9
    assert max(ratio(p, q) for p in range(P) for q in range(P) if p != q) < 0.4


def test_full_rank_channel_propagation_equals_full(k2):
    m, K = k2
    Nk = m.p.L ** 2
    D, U, S, V = oc.channel_svd(K, m.p.Nb, Nk)
    pulse = wl.Pulse(E0=0.01, omega=0.12, t0=8.0, sigma=4.0)
    s = op.half_step_samples(pulse, 0.2, 60)
    full, _ = op.rk4(m, lambda v: K @ v, s, 0.2, 60)
    ch, _ = op.rk4(m, lambda v: oc.apply_channel(D, U, S, V, v), s, 0.2, 60)
    assert op.rel_l2(ch[:, 0], full[:, 0]) < 1e-11
