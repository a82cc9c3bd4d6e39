"""Pins of the oracle's dense linear algebra and angle selection (reading
R8) against numpy / LAPACK and brute force."""
import itertools

import numpy as np
import pytest
import scipy.linalg


def _rand(m, n, seed):
    return np.random.default_rng(seed).standard_normal((m, n))


def test_lu_solve_matches_numpy(orc):
    A = _rand(9, 9, 1)
    B = _rand(9, 3, 2)
    np.testing.assert_allclose(orc.lu_solve(A, B), np.linalg.solve(A, B), rtol=1e-12, atol=1e-13)


def test_householder_qr_matches_numpy(orc):
    A = _rand(50, 7, 3)
    Q, R = orc.householder_qr(A)
    Qn, Rn = np.linalg.qr(A)
    sgn = np.sign(np.diag(Rn))
    np.testing.assert_allclose(Q, Qn * sgn, atol=1e-13)
    np.testing.assert_allclose(R, Rn * sgn[:, None], atol=1e-13)
    assert np.all(np.diag(R) >= 0)
    np.testing.assert_allclose(Q.T @ Q, np.eye(7), atol=1e-14)


def test_householder_qr_rank_deficient(orc):
    A = _rand(20, 5, 4)
    A[:, 2] = 0.0
    A[:, 4] = A[:, 1]
    Q, R = orc.householder_qr(A)
    np.testing.assert_allclose(Q.T @ Q, np.eye(5), atol=1e-14)
    np.testing.assert_allclose(Q @ R, A, atol=1e-13)


def test_jacobi_svd_matches_numpy(orc):
    A = _rand(8, 8, 5)
    U, s, V = orc.jacobi_svd(A)
    np.testing.assert_allclose(s, np.linalg.svd(A, compute_uv=False), rtol=1e-13)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(8), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(8), atol=1e-13)


def test_jacobi_svd_rank_deficient(orc):
    B = _rand(6, 3, 6)
    A = B @ _rand(3, 6, 7)
    U, s, V = orc.jacobi_svd(A)
    np.testing.assert_allclose(s[:3], np.linalg.svd(A, compute_uv=False)[:3], rtol=1e-12)
    assert np.all(s[3:] < 1e-13 * s[0])
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-12)
    np.testing.assert_allclose(U @ np.diag(s) @ V.T, A, atol=1e-12)


def _orthonormal(n, r, seed):
    Q, _ = np.linalg.qr(_rand(n, r, seed))
    return Q


@pytest.mark.parametrize("n,r,seed", [(64, 8, 10), (128, 16, 11), (200, 5, 12)])
def test_qdeim_matches_lapack_dgeqp3(orc, n, r, seed):
    W = _orthonormal(n, r, seed)
    _, _, piv = scipy.linalg.qr(W.T, pivoting=True, mode="economic")  # LAPACK dgeqp3
    assert list(orc.qdeim(W)) == list(piv[:r])


@pytest.mark.parametrize("n,r,seed", [(8, 2, 20), (10, 3, 21), (12, 3, 22)])
def test_qdeim_is_greedy_max_volume(orc, n, r, seed):
    W = _orthonormal(n, r, seed)
    idx = list(orc.qdeim(W))
    for s in range(r):
        prev = idx[:s]
        vols = {}
        for k in range(n):
            if k in prev:
                continue
            M = W[prev + [k], :]
            vols[k] = np.linalg.det(M @ M.T)
        assert idx[s] == max(vols, key=vols.get)
    # within the pivoted-QR volume bound of the brute-force maximum
    best = max(abs(np.linalg.det(W[list(c), :])) for c in itertools.combinations(range(n), r))
    got = abs(np.linalg.det(W[idx, :]))
    assert got >= best / (np.sqrt(n - r + 1) * 2 ** r)


def test_qdeim_tie_rule_lowest_index(orc):
    # duplicated rows: the tie goes to the lower index
    W = _orthonormal(10, 3, 30)
    W = np.vstack([W, W])
    idx = orc.qdeim(W)
    assert np.all(idx < 10)


def test_deim_interpolation_property(orc):
    W = _orthonormal(40, 6, 40)
    idx = list(orc.deim(W))
    assert len(set(idx)) == 6
    assert idx[0] == int(np.argmax(np.abs(W[:, 0])))
    for j in range(1, 6):
        c = np.linalg.solve(W[idx[:j], :j], W[idx[:j], j])
        res = W[:, j] - W[:, :j] @ c
        np.testing.assert_allclose(res[idx[:j]], 0.0, atol=1e-13)
        assert idx[j] == int(np.argmax(np.abs(res)))
    # r = 1: DEIM and pivoted QR coincide
    assert orc.deim(W[:, :1])[0] == orc.qdeim(W[:, :1])[0]


def test_beta_What_inverse_constant_is_4pi(orc):
    # appendix identity: beta^T What^{-1} [1] = 4 pi when 1 is in span W
    p = orc.Problem(4, 4, 8, 16, np.ones(16), np.ones(16))
    X0, S0, W0 = orc.initial_factors(p, np.full(16, 0.3), 10)
    ox, oy, oz, w = orc.quadrature(8, 16)
    beta = w @ W0
    for idx in (orc.qdeim(W0), orc.deim(W0)):
        val = beta @ np.linalg.solve(W0[idx, :], np.ones(10))
        assert abs(val - 4 * np.pi) < 1e-12
