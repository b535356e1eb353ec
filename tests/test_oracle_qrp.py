"""Pins for the oracle's Householder QR with column pivoting (Section III-D).

Checked against a hand-worked reflector, LAPACK's dgeqp3 (scipy), and the
properties the section states: A P = Q R, Q orthonormal, R upper triangular with
non-increasing |r_jj|."""

import numpy as np
import pytest
import scipy.linalg

import oracle


def test_single_reflector_by_hand():
    # x = (3, 4): ||x|| = 5, v = x + sign(3)*5*e1 = (8, 4), H x = (-5, 0),
    # Q e1 = H e1 = (1 - 2*64/80, -2*32/80) = (-0.6, -0.8).
    res = oracle.qrp(np.array([[3.0], [4.0]]), 1)
    assert res.piv.tolist() == [0]
    assert res.rdiag[0] == pytest.approx(-5.0, abs=1e-15)
    np.testing.assert_allclose(res.Q[:, 0], [-0.6, -0.8], atol=1e-15)


def test_sign_of_zero_is_plus_one():
    # a_jj = 0: v = x + (+1)||x|| e1 = (2, 2), so r_jj = -||x|| = -2 and
    # Q e1 = e1 - 2 v v_1 / (v^T v) = (1 - 8/8, -8/8) = (0, -1).
    res = oracle.qrp(np.array([[0.0], [2.0]]), 1)
    assert res.rdiag[0] == pytest.approx(-2.0, abs=1e-15)
    np.testing.assert_allclose(res.Q[:, 0], [0.0, -1.0], atol=1e-15)


def test_pivot_order_by_hand():
    # columns with norms 1, 3, 2 (mutually orthogonal): pivots 1, 2, 0.
    A = np.array([[1.0, 0, 0], [0, 3.0, 0], [0, 0, 2.0], [0, 0, 0]])
    res = oracle.qrp(A, 3)
    assert res.piv.tolist() == [1, 2, 0]
    np.testing.assert_allclose(np.abs(res.rdiag), [3.0, 2.0, 1.0], atol=1e-15)


def test_ties_take_smallest_index():
    A = np.array([[1.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    res = oracle.qrp(A, 2)
    assert res.piv[0] == 0


def _r_block(A, res):
    return res.Q.T @ A[:, res.piv]


@pytest.mark.parametrize("m,n,k", [(40, 12, 12), (40, 12, 5), (12, 12, 7), (9, 30, 9), (50, 3, 3)])
def test_properties(m, n, k):
    rng = np.random.default_rng(m * 100 + n + k)
    A = rng.standard_normal((m, n)) * rng.uniform(0.1, 10.0, n)
    res = oracle.qrp(A, k)
    Q = res.Q
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-13)
    Rk = _r_block(A, res)                       # k x k block of R on the pivoted columns
    np.testing.assert_allclose(np.tril(Rk, -1), 0.0, atol=1e-12 * np.abs(A).max())
    np.testing.assert_allclose(np.diag(Rk), res.rdiag, rtol=1e-12, atol=1e-12)
    # the pivoted columns lie in span(Q_k): A P_k = Q_k R_k
    np.testing.assert_allclose(Q @ Rk, A[:, res.piv], atol=1e-12 * np.abs(A).max())
    d = np.abs(res.rdiag)
    assert np.all(d[:-1] >= d[1:] - 1e-12 * d[0])


@pytest.mark.parametrize("m,n", [(60, 10), (25, 25), (80, 16)])
def test_matches_lapack_dgeqp3(m, n):
    rng = np.random.default_rng(m + 7 * n)
    # well separated column scales keep every pivot decision far from a tie
    scales = 2.0 ** (-np.arange(n) * 1.5)
    A = rng.standard_normal((m, n)) * rng.permutation(scales)
    k = min(m, n)
    res = oracle.qrp(A, k)
    Ql, Rl, Pl = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert res.piv.tolist() == Pl[:k].tolist()
    np.testing.assert_allclose(np.abs(res.rdiag), np.abs(np.diag(Rl))[:k], rtol=1e-10)
    signs = np.sign(np.sum(res.Q * Ql[:, :k], axis=0))
    np.testing.assert_allclose(res.Q, Ql[:, :k] * signs, atol=1e-10)


def test_rank_deficient_no_nan():
    rng = np.random.default_rng(2)
    B = rng.standard_normal((20, 2))
    A = B @ rng.standard_normal((2, 6))        # rank 2
    res = oracle.qrp(A, 4)
    assert np.all(np.isfinite(res.Q)) and np.all(np.isfinite(res.rdiag))
    assert abs(res.rdiag[2]) < 1e-12 * abs(res.rdiag[0])
    np.testing.assert_allclose(res.Q.T @ res.Q, np.eye(4), atol=1e-12)


def test_exact_zero_column_gives_identity_reflector():
    A = np.zeros((5, 3))
    A[:, 0] = [1, 2, 0, 0, 0]
    res = oracle.qrp(A, 2)
    assert res.rdiag[1] == 0.0
    np.testing.assert_allclose(res.Q.T @ res.Q, np.eye(2), atol=1e-15)


def test_fat_case_runs_on_gram():
    rng = np.random.default_rng(9)
    Y = rng.standard_normal((6, 3)) @ rng.standard_normal((3, 20))  # 6 x 20, rank 3
    S = oracle.gram(Y)
    np.testing.assert_allclose(S, Y @ Y.T, rtol=1e-13, atol=1e-12)
    res = oracle.qrp_factor(Y, 3)
    U = res.Q
    # span(U) = column space of Y: projecting Y onto it loses nothing
    np.testing.assert_allclose(U @ (U.T @ Y), Y, atol=1e-10 * np.abs(Y).max())
    direct = oracle.qrp_factor(Y, 3, direct=True)
    P1, P2 = U @ U.T, direct.Q @ direct.Q.T
    np.testing.assert_allclose(P1, P2, atol=1e-10)


def test_rejects_k_above_min_dim():
    with pytest.raises(ValueError):
        oracle.qrp(np.ones((3, 5)), 4)
