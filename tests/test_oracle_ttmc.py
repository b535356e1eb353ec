"""Pins for the oracle's COO handling and sparse TTMc (Algorithm 2 inner loop).

The oracle's TTMc is a per-nonzero Kronecker accumulation; these tests check it
against things that do not share that formula: a dense mode-product chain (the
power-iteration TTM of eq. power_ite), the hand-worked Table I example, and the
Kronecker-product count printed for the PMM tensor."""

import os

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth


def dense_of(dims, coords, vals):
    X = np.zeros(dims, dtype=np.float64)
    np.add.at(X, tuple(coords.astype(np.int64)), np.asarray(vals, dtype=np.float64))
    return X


def dense_ttm_chain(X, U, mode):
    """Y = X x_1 U_1^T ... (skip mode) ... x_N U_N^T, unfolded with the mode first and the
    remaining rank indices in C order (last fastest)."""
    Y = X
    N = X.ndim
    for m in range(N):
        if m == mode:
            continue
        Y = np.tensordot(Y, U[m], axes=([m], [0]))  # contracted axis replaced at the end
        Y = np.moveaxis(Y, -1, m)
    Y = np.moveaxis(Y, mode, 0)
    return Y.reshape(X.shape[mode], -1)


def random_coo(rng, dims, nnz, dup_frac=0.2):
    coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    ndup = int(nnz * dup_frac)
    if ndup:
        src = rng.integers(0, nnz, ndup)
        dst = rng.integers(0, nnz, ndup)
        coords[:, dst] = coords[:, src]
    vals = rng.standard_normal(nnz)
    return coords, vals


@pytest.mark.parametrize("dims,ranks", [((6, 5, 4), (2, 3, 2)), ((4, 3, 3, 2), (2, 2, 3, 2)),
                                        ((7, 9), (3, 4)), ((3, 4, 2, 3, 2), (2, 1, 2, 3, 2))])
def test_ttmc_matches_dense_mode_products(dims, ranks):
    rng = np.random.default_rng(7)
    coords, vals = random_coo(rng, dims, 40)
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    X = dense_of(dims, coords, vals)
    for n in range(len(dims)):
        Y = oracle.ttmc(dims, ranks, coords, vals, n, U)
        ref = dense_ttm_chain(X, U, n)
        assert Y.shape == ref.shape
        np.testing.assert_allclose(Y, ref, rtol=1e-13, atol=1e-13 * np.abs(ref).max())


def test_ttmc_does_not_read_own_factor():
    rng = np.random.default_rng(3)
    dims, ranks = (5, 6, 7), (2, 3, 2)
    coords, vals = random_coo(rng, dims, 30)
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    for n in range(3):
        U2 = list(U)
        U2[n] = np.full_like(U[n], np.nan)
        np.testing.assert_array_equal(oracle.ttmc(dims, ranks, coords, vals, n, U),
                                      oracle.ttmc(dims, ranks, coords, vals, n, U2))


def load_table1(golden_dir):
    coo, ys = [], []
    with open(os.path.join(golden_dir, "table1_ttmc.txt")) as f:
        for line in f:
            t = line.split()
            if not t or t[0].startswith("#"):
                continue
            if t[0] == "coo":
                coo.append([int(v) for v in t[1:5]] + [float(t[5])])
            elif t[0] == "y":
                ys.append((int(t[1]) - 1, int(t[2]), [float(v) for v in t[3:]]))
    return coo, ys


def test_ttmc_table1_worked_example(golden_dir):
    coo, ys = load_table1(golden_dir)
    coords = np.array([[c[m] - 1 for c in coo] for m in range(4)], dtype=np.uint32)
    vals = np.array([c[4] for c in coo])
    dims, ranks = (5, 5, 5, 5), (2, 2, 2, 2)
    U = [np.stack([np.ones(5), np.arange(1, 6)], axis=1) for _ in range(4)]
    expected = {n: np.zeros((5, 8)) for n in range(4)}
    for n, row, v in ys:
        expected[n][row] = v
    for n in range(4):
        np.testing.assert_array_equal(oracle.ttmc(dims, ranks, coords, vals, n, U), expected[n])


def test_coalesce_sums_duplicates():
    rng = np.random.default_rng(11)
    dims = (4, 3, 5)
    coords, vals = random_coo(rng, dims, 60, dup_frac=0.5)
    cc, cv = oracle.coalesce(coords, vals)
    ref = {}
    for z in range(coords.shape[1]):
        key = tuple(int(c) for c in coords[:, z])
        ref[key] = ref.get(key, 0.0) + vals[z]
    keys = sorted(ref)
    assert cc.shape == (3, len(keys))
    assert [tuple(int(c) for c in cc[:, z]) for z in range(cc.shape[1])] == keys
    np.testing.assert_allclose(cv, [ref[k] for k in keys], rtol=1e-15, atol=1e-15)
    # the norm of the coalesced tensor equals the dense Frobenius norm (Definition 2)
    assert oracle.norm2(cv) == pytest.approx(np.sum(dense_of(dims, coords, vals) ** 2), rel=1e-14)


def test_pmm_tensor_and_kronecker_count(golden_dir):
    spec = {}
    with open(os.path.join(golden_dir, "pmm_counts.txt")) as f:
        for line in f:
            t = line.split()
            if t and not t[0].startswith("#"):
                spec[t[0]] = t[1:]
    dims, coords, vals = synth.pmm_tensor(5, 5, 5)
    assert list(dims) == [int(v) for v in spec["dims"]]
    assert coords.shape[1] == int(spec["nnz"][0])
    assert coords.shape[1] / np.prod(dims) == pytest.approx(float(spec["sparsity"][0]))
    # PMM is binary: one entry per scalar product, no duplicates
    assert oracle.coalesce(coords, vals)[1].shape[0] == coords.shape[1]
    ranks = tuple(int(v) for v in spec["ranks"])
    sweeps = int(spec["sweeps"][0])
    rng = np.random.default_rng(5)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    oracle.kron_reset()
    res = oracle.hooi(dims, ranks, coords, vals, U0, sweeps)
    assert oracle.kron_count() == int(spec["kronecker_products"][0])
    assert all(0.0 <= f <= 1.0 for f in res.fits)
