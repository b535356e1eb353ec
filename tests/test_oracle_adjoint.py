"""Pins for the oracle's observed-entry loss and gradients (the differentiation form).

The loss is checked against a dense reconstruction [[G; U_1..U_N]] evaluated at the
observed coordinates, and every gradient against central finite differences of
that loss in FP64."""

import numpy as np
import pytest

import oracle
from tests.test_oracle_hooi import reconstruct


def dense_loss(dims, coords, vals, U, G):
    Xh = reconstruct(G, U)
    e = Xh[tuple(coords.astype(np.int64))] - vals
    return 0.5 * float(np.sum(e * e))


@pytest.mark.parametrize("dims,ranks", [((5, 6, 4), (2, 3, 2)), ((4, 3, 3, 5), (2, 2, 3, 2)), ((6, 7), (3, 2))])
def test_loss_and_gradients_by_finite_differences(dims, ranks):
    rng = np.random.default_rng(sum(dims))
    nnz = 25
    coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    vals = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    G = rng.standard_normal(ranks)
    L, dU, dG = oracle.loss_grad(dims, ranks, coords, vals, U, G)
    assert L == pytest.approx(dense_loss(dims, coords, vals, U, G), rel=1e-13)
    h = 1e-6
    for m in range(len(dims)):
        for _ in range(6):
            i, r = rng.integers(0, dims[m]), rng.integers(0, ranks[m])
            Up = [u.copy() for u in U]
            Um = [u.copy() for u in U]
            Up[m][i, r] += h
            Um[m][i, r] -= h
            fd = (dense_loss(dims, coords, vals, Up, G) - dense_loss(dims, coords, vals, Um, G)) / (2 * h)
            assert dU[m][i, r] == pytest.approx(fd, rel=1e-6, abs=1e-7)
    for _ in range(8):
        idx = tuple(rng.integers(0, r) for r in ranks)
        Gp, Gm = G.copy(), G.copy()
        Gp[idx] += h
        Gm[idx] -= h
        fd = (dense_loss(dims, coords, vals, U, Gp) - dense_loss(dims, coords, vals, U, Gm)) / (2 * h)
        assert dG[idx] == pytest.approx(fd, rel=1e-6, abs=1e-7)


def test_gradient_of_G_is_a_ttmc_of_the_residual():
    # dL/dG = E x_1 U_1^T ... x_N U_N^T where E holds the residuals at the observed
    # coordinates; written through the dense TTM chain this is independent of the
    # oracle's per-nonzero loops.
    rng = np.random.default_rng(3)
    dims, ranks = (5, 4, 6), (2, 3, 2)
    nnz = 30
    coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    vals = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    G = rng.standard_normal(ranks)
    _, dU, dG = oracle.loss_grad(dims, ranks, coords, vals, U, G)
    Xh = reconstruct(G, U)
    E = np.zeros(dims)
    np.add.at(E, tuple(coords.astype(np.int64)), Xh[tuple(coords.astype(np.int64))] - vals)
    ref = E
    for m in range(3):
        ref = np.moveaxis(np.tensordot(ref, U[m], axes=([m], [0])), -1, m)
    np.testing.assert_allclose(dG, ref, rtol=1e-12, atol=1e-12)
    # dL/dU_1 = E_(1) (U_2 kron U_3) G_(1)^T
    Y = np.moveaxis(np.tensordot(np.tensordot(E, U[1], axes=([1], [0])), U[2], axes=([1], [0])), 0, 0)
    ref1 = Y.reshape(dims[0], -1) @ G.reshape(ranks[0], -1).T
    np.testing.assert_allclose(dU[0], ref1, rtol=1e-12, atol=1e-12)
