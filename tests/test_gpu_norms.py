"""The column sums of squares of Y_(n) that the pipelined FP32 TTMc forms as it writes
Y_(n) (ttmc_mode_norms), and their use as the initial pivot norms of the QRP inside
hooi_iter (Section III-D: the pivot is the column of largest remaining norm).

- The norms are those of the Y the TTMc wrote: exact FP32 squares summed in double-float
  pairs, so within 1e-12 (relative) of the FP64 sums of squares of that Y.
- Against the oracle's FP64 Y: each column within 3e-5 of its squared norm (twice the
  FP32 TTMc's 1e-5 bar, plus a floor of 1e-9 of the largest column for tiny columns).
- HOOI whose QRP takes these norms (TUCKER_F_TTMC_NORMS) against HOOI whose QRP forms its
  own, from the same start.  After one sweep U_1 (the QRP of the same Y_(1)) within 1e-9: the
  two differ only in the initial norms' summation order and in the offsets of the A^T y
  sums.  Later modes see FP32 copies of factors that may round differently, so over three
  sweeps the bar is the FP32 one: fits within 1e-9, subspace projectors within 1e-5; and
  the oracle's fits within 1e-6."""
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, torch
from tests.test_gpu_ttmc import draw, oracle_all_modes

pytestmark = pytest.mark.gpu

CASES = [
    # (name, dims, ranks, nnz, coord recipe): several blocks of work units and a ragged tail
    ("r16-uniform", (300, 250, 40), (16, 16, 16), 70_003, "uniform"),
    ("r16-zipf", (2000, 1500, 900), (16, 16, 16), 60_001, "zipf"),
    ("r8", (100, 100, 100), (8, 8, 8), 10_000, "distinct"),
    ("r16-r8", (200, 300, 150), (8, 16, 8), 30_001, "uniform"),
    ("r8-r16", (90, 20, 200), (8, 8, 16), 25_013, "uniform"),
    ("long-slices", (5, 3000, 2000), (4, 16, 16), 50_000, "uniform"),
    ("long-fibers", (60, 16, 500), (16, 16, 16), 40_009, "uniform"),
]


# (rank of the first, of the second remaining mode) of the pipelined form with P_n <= 256
PIPE_SHAPES = {(16, 16), (8, 8), (16, 8), (8, 16)}


@pytest.mark.parametrize("fibers", ["1", "0"], ids=["fibers", "nonzeros"])
@pytest.mark.parametrize("chunk", [None, "32"], ids=["default-units", "small-units"])
@pytest.mark.parametrize("name,dims,ranks,nnz,recipe", CASES, ids=[c[0] for c in CASES])
def test_norms_of_the_written_y(name, dims, ranks, nnz, recipe, chunk, fibers, monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", fibers)
    if chunk:
        monkeypatch.setenv("TUCKER_TTMC_CHUNK", chunk)
    T = lib()
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    coords = draw(rng, dims, nnz, recipe)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx = T.tucker_init(dims, torch.as_tensor(coords.astype(np.int32)).cuda(),
                        torch.as_tensor(vals).cuda(), ranks, [torch.as_tensor(u).cuda() for u in U])
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        other = tuple(ranks[m] for m in range(3) if m != n)
        if other not in PIPE_SHAPES:  # another TTMc form: no norms
            with pytest.raises(T.TuckerError, match="TUCKER_EINVAL"):
                T.ttmc_mode_norms(ctx, n)
            continue
        Y, cs = T.ttmc_mode_norms(ctx, n)
        Y = Y.cpu().numpy().astype(np.float64)
        cs = cs.cpu().numpy()
        own = (Y * Y).sum(axis=0)
        np.testing.assert_allclose(cs, own, rtol=1e-12, atol=1e-300)
        # the same Y as ttmc_mode, bit for bit
        np.testing.assert_array_equal(T.ttmc_mode(ctx, n).cpu().numpy(), Y.astype(np.float32))
        want = (ref[n] * ref[n]).sum(axis=0)
        np.testing.assert_allclose(cs, want, rtol=3e-5, atol=1e-9 * want.max())


def test_norms_refused_where_not_formed():
    """BF16 factors, an order-4 tensor and P_n > 256 run other TTMc forms: EINVAL, with Y
    still written."""
    T = lib()
    rng = np.random.default_rng(5)
    for dims, ranks, kw in [((60, 50, 40), (8, 8, 8), {"bf16": True}),
                            ((30, 20, 10, 8), (4, 4, 4, 4), {}),
                            ((40, 32, 100), (32, 32, 32), {})]:
        nnz = 5000
        coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.int32)
        vals = rng.standard_normal(nnz).astype(np.float32)
        ctx = T.tucker_init(dims, torch.as_tensor(coords).cuda(), torch.as_tensor(vals).cuda(), ranks, **kw)
        with pytest.raises(T.TuckerError, match="TUCKER_EINVAL"):
            T.ttmc_mode_norms(ctx, 0)


def gpu_sweeps(w, iters, **kw):
    """Fits of `iters` sweeps, U_1 after the first, all factors after the last, launches."""
    T = lib()
    dims, ranks = w.workload.dims, w.workload.ranks
    ctx = T.tucker_init(dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(),
                        ranks, [torch.as_tensor(u).cuda() for u in w.U0], **kw)
    torch.cuda.synchronize()
    l0 = T.tucker_kernel_launches()
    fits = [T.hooi_iter(ctx)]
    U1 = T.tucker_get_factor(ctx, 0).cpu().numpy()
    fits += [T.hooi_iter(ctx) for _ in range(iters - 1)]
    launches = T.tucker_kernel_launches() - l0
    U = [T.tucker_get_factor(ctx, n).cpu().numpy() for n in range(len(dims))]
    return fits, U1, U, launches


@pytest.mark.parametrize("fibers", ["1", "0"], ids=["fibers", "nonzeros"])
def test_hooi_with_ttmc_norms(fibers, monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", fibers)
    wl = synth.Workload("skew-small", (3000, 3000, 200), 400_000, (16, 16, 16), 3, 91,
                        (("zipf", 1.2), ("uniform",), ("uniform",)), "lognormal")
    w = synth.make(wl)
    fits, U1, U, launches = gpu_sweeps(w, 3, ttmc_norms=True)
    fits_own, U1_own, U_own, launches_own = gpu_sweeps(w, 3)
    # one norm reduction per sweep on each mode whose QRP runs on Y_(n) itself (I_n >= P_n;
    # the last mode, 200 x 256, goes through Y Y^T and forms none)
    assert launches - launches_own == 3 * 2
    assert float(np.max(np.abs(U1 - U1_own))) <= 1e-9
    np.testing.assert_allclose(fits, fits_own, rtol=0, atol=1e-9)
    for n in range(3):
        assert np.linalg.norm(U[n] @ U[n].T - U_own[n] @ U_own[n].T) <= 1e-5 * np.sqrt(wl.ranks[n])
    ref = oracle.hooi(wl.dims, wl.ranks, w.coords, w.vals.astype(np.float64), w.U0, 3,
                      threads=os.cpu_count() or 1)
    np.testing.assert_allclose(fits, ref.fits, rtol=0, atol=1e-6)
