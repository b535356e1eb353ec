"""The column-split oracle routines (tucker_oracle_par.c, used to time the oracle on all
host cores) against the serial oracle: equal bit for bit, since every output entry is
computed with the serial routine's operations in the serial order."""
import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth


@pytest.mark.parametrize("dims,ranks,nnz,threads", [((30, 40, 50), (4, 5, 6), 3000, 4), ((9, 8, 7, 6), (2, 3, 2, 3), 800, 3),
                                                   ((60, 50), (5, 7), 1000, 7), ((20, 20, 20), (8, 8, 8), 2000, 16)])
def test_ttmc_split_by_columns_equals_serial(dims, ranks, nnz, threads):
    rng = np.random.default_rng(nnz + threads)
    coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    vals = rng.standard_normal(nnz)
    U = [rng.standard_normal((d, r)) for d, r in zip(dims, ranks)]
    for n in range(len(dims)):
        a = oracle.ttmc(dims, ranks, coords, vals, n, U)
        b = oracle.ttmc(dims, ranks, coords, vals, n, U, threads=threads)
        assert np.array_equal(a, b)


@pytest.mark.parametrize("m,n,k,threads", [(200, 64, 16, 4), (50, 300, 20, 5), (120, 33, 33, 8), (7, 3, 3, 2)])
def test_qrp_gram_core_split_equal_serial(m, n, k, threads):
    rng = np.random.default_rng(m + n + k)
    A = rng.standard_normal((m, n)) * rng.uniform(0.2, 5.0, n)
    A[:, n // 2] = 0.0
    r1, r2 = oracle.qrp(A, k), oracle.qrp(A, k, threads=threads)
    assert np.array_equal(r1.Q, r2.Q) and np.array_equal(r1.piv, r2.piv) and np.array_equal(r1.rdiag, r2.rdiag)
    assert np.array_equal(oracle.gram(A), oracle.gram(A, threads))
    U = rng.standard_normal((m, 3))
    assert np.array_equal(oracle.core(A, U, (n, 3)), oracle.core(A, U, (n, 3), threads))


def test_hooi_split_equals_serial_on_the_tiny_recipe():
    w = synth.make("tiny-100^3")
    a = oracle.hooi(w.workload.dims, w.workload.ranks, w.coords, w.vals.astype(np.float64), w.U0, 3)
    b = oracle.hooi(w.workload.dims, w.workload.ranks, w.coords, w.vals.astype(np.float64), w.U0, 3, threads=6)
    assert a.fits == b.fits
    assert np.array_equal(a.G, b.G)
    for x, y in zip(a.U, b.U):
        assert np.array_equal(x, y)
