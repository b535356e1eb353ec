"""Pins for the oracle's core tensor, fit and HOOI sweep (Algorithm 2)."""

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.test_oracle_ttmc import dense_of, random_coo


def full_projection(X, U):
    G = X
    for m in range(X.ndim):
        G = np.tensordot(G, U[m], axes=([m], [0]))
        G = np.moveaxis(G, -1, m)
    return G


def reconstruct(G, U):
    X = G
    for m in range(G.ndim):
        X = np.tensordot(X, U[m], axes=([m], [1]))
        X = np.moveaxis(X, -1, m)
    return X


@pytest.mark.parametrize("dims,ranks", [((6, 5, 4), (2, 3, 2)), ((4, 3, 5, 2), (2, 2, 3, 2)), ((7, 9), (3, 4))])
def test_core_matches_full_projection(dims, ranks):
    rng = np.random.default_rng(1)
    coords, vals = random_coo(rng, dims, 50)
    U = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    N = len(dims)
    Y = oracle.ttmc(dims, ranks, coords, vals, N - 1, U)
    G = oracle.core(Y, U[N - 1], ranks)
    X = dense_of(dims, coords, vals)
    ref = full_projection(X, U)
    np.testing.assert_allclose(G, ref, rtol=1e-12, atol=1e-13 * np.abs(ref).max())
    assert np.sum(G ** 2) <= np.sum(X ** 2) * (1 + 1e-12)


def test_fit_from_core_equals_dense_residual():
    rng = np.random.default_rng(4)
    dims, ranks = (6, 7, 5), (3, 2, 3)
    coords, vals = random_coo(rng, dims, 80, dup_frac=0.0)
    cc, cv = oracle.coalesce(coords, vals)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    res = oracle.hooi(dims, ranks, cc, cv, U0, 2, coalesced=True)
    X = dense_of(dims, cc, cv)
    Xh = reconstruct(res.G, res.U)
    direct = 1.0 - np.linalg.norm(X - Xh) / np.linalg.norm(X)
    assert res.fits[-1] == pytest.approx(direct, abs=1e-12)


@pytest.mark.parametrize("svd", [False, True])
def test_exact_recovery_of_known_tucker_rank(svd):
    rng = np.random.default_rng(12)
    dims, ranks = (12, 10, 8), (3, 3, 2)
    X, coords, vals = synth.low_rank_dense(rng, dims, ranks)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    res = oracle.hooi(dims, ranks, coords, vals, U0, 2, svd=svd)
    # ||X||^2 - ||G||^2 is an O(eps ||X||^2) difference under a square root
    assert res.fits[-1] > 1.0 - 1e-6
    np.testing.assert_allclose(reconstruct(res.G, res.U), X, atol=1e-10 * np.abs(X).max())
    for u in res.U:
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)


def test_qrp_and_svd_reach_the_same_fit_on_low_rank_data():
    # Table II analogue: QRP-HOOI is as accurate as SVD-HOOI on low-rank tensors.
    rng = np.random.default_rng(21)
    dims, ranks = (10, 9, 8, 6), (2, 3, 2, 2)
    X, coords, vals = synth.low_rank_dense(rng, dims, ranks)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    a = oracle.hooi(dims, ranks, coords, vals, U0, 2)
    b = oracle.hooi(dims, ranks, coords, vals, U0, 2, svd=True)
    assert a.fits[-1] == pytest.approx(b.fits[-1], abs=1e-6)


def test_svd_mode_fit_is_monotone():
    rng = np.random.default_rng(8)
    dims, ranks = (15, 12, 10), (3, 3, 3)
    coords, vals = random_coo(rng, dims, 300, dup_frac=0.0)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    res = oracle.hooi(dims, ranks, coords, vals, U0, 6, svd=True)
    f = np.array(res.fits)
    assert np.all(f[1:] >= f[:-1] - 1e-12)
    assert np.all((0 <= f) & (f <= 1))


def test_factor_orthonormality_and_fit_range_qrp():
    rng = np.random.default_rng(31)
    dims, ranks = (20, 18, 16), (4, 4, 4)
    coords, vals = random_coo(rng, dims, 500)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    res = oracle.hooi(dims, ranks, coords, vals, U0, 3)
    for u in res.U:
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-13)
    assert all(0.0 <= f <= 1.0 for f in res.fits)


def test_fat_unfolding_uses_gram_branch():
    # mode-1 unfolding is 3 x 16 (P > I): the paper runs QRP on Y Y^T there.
    rng = np.random.default_rng(17)
    dims, ranks = (3, 6, 5), (2, 4, 4)
    coords, vals = random_coo(rng, dims, 60, dup_frac=0.0)
    cc, cv = oracle.coalesce(coords, vals)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    res = oracle.hooi(dims, ranks, cc, cv, U0, 1, coalesced=True)
    Y = oracle.ttmc(dims, ranks, cc, cv, 0, U0)
    assert Y.shape == (3, 16)
    np.testing.assert_allclose(res.U[0], oracle.qrp(Y @ Y.T, 2).Q, atol=1e-12)
    assert not np.allclose(res.U[0], oracle.qrp(Y, 2).Q)
