"""GPU parity of the fiber form of the TTMc (order 3, Section III-C: the nonzeros of a
slice that share the index of the first remaining mode form a fiber whose factor sum is
formed once) against the FP64 oracle, with the form forced on and off at init.

Inputs are chosen so that fibers are long (small middle dimensions, Zipf indices),
longer than the 32-nonzero cut, and so that slices are split over several work units
(small unit size); the relative Frobenius bar is the FP32 one, 1e-5."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import rel_fro
from tests.test_gpu_ttmc import draw, oracle_all_modes, run_ttmc_all_modes

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    # (name, dims, ranks, nnz, coord recipe)
    ("long-fibers-r16", (60, 16, 500), (16, 16, 16), 40_009, "uniform"),
    ("zipf-r16", (3000, 2000, 400), (16, 16, 16), 80_021, "zipf"),
    ("r8", (100, 12, 90), (8, 8, 8), 30_011, "uniform"),
    ("r16-r8", (80, 16, 300), (16, 16, 8), 25_003, "uniform"),
    ("r8-r16", (90, 20, 200), (8, 8, 16), 25_013, "uniform"),
    ("r32", (40, 32, 100), (32, 32, 32), 12_007, "uniform"),
    ("dense-ish", (30, 30, 30), (16, 16, 16), 20_000, "distinct"),
    ("single-slice", (1, 50, 400), (1, 16, 16), 20_011, "uniform"),
    # mode 1's slices repeat the index of mode 3 far more than that of mode 2: its copy is
    # re-sorted so that mode 3 is the middle level
    ("middle-last-r16-r8", (60, 2000, 12), (16, 16, 8), 40_009, "uniform"),
    ("middle-last-r16", (50, 3000, 16), (16, 16, 16), 30_011, "uniform"),
]


@pytest.fixture(params=["1", "0"], ids=["fibers", "nonzeros"])
def fiber_policy(request, monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", request.param)
    return request.param


@pytest.mark.parametrize("chunk", [None, "32"], ids=["default-units", "small-units"])
@pytest.mark.parametrize("name,dims,ranks,nnz,recipe", CASES, ids=[c[0] for c in CASES])
def test_fiber_form_matches_oracle(name, dims, ranks, nnz, recipe, chunk, fiber_policy, monkeypatch):
    if chunk:
        monkeypatch.setenv("TUCKER_TTMC_CHUNK", chunk)
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    coords = draw(rng, dims, nnz, recipe)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        err = rel_fro(Ys[n], ref[n])
        assert err <= TOL, f"mode {n}: relative Frobenius error {err:.3e}"
        np.testing.assert_allclose(Ys[n], ref[n], rtol=0, atol=TOL * np.abs(ref[n]).max())


def test_fiber_form_empty_rows_and_duplicates(fiber_policy):
    # rows 3 and 7 of mode 0 are empty; duplicates are summed before the fibers are formed
    rng = np.random.default_rng(17)
    dims, ranks = (10, 16, 50), (8, 8, 8)
    coords = np.stack([rng.choice([0, 1, 2, 4, 5, 6, 8, 9], 3000), rng.integers(0, 16, 3000),
                       rng.integers(0, 50, 3000)]).astype(np.uint32)
    coords = np.concatenate([coords, coords[:, :500]], axis=1)
    vals = rng.standard_normal(coords.shape[1]).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    np.testing.assert_array_equal(Ys[0][[3, 7]], 0.0)
    for n in range(3):
        assert rel_fro(Ys[n], ref[n]) <= TOL


def test_fiber_form_is_deterministic(monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", "1")
    rng = np.random.default_rng(23)
    dims, ranks = (500, 30, 400), (16, 16, 16)
    coords = draw(rng, dims, 60_000, "zipf")
    vals = rng.standard_normal(60_000).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    _, Y1 = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    _, Y2 = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    for a, b in zip(Y1, Y2):
        np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("dims", [(40, 8, 60), (40, 60, 8)], ids=["middle-first", "middle-last"])
def test_fiber_form_in_the_adjoint(monkeypatch, dims):
    """The loss gradient runs the TTMc of the residual tensor through the same form
    (including a mode whose copy is re-sorted for its fiber level)."""
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", "1")
    from tests.test_gpu_adjoint import gpu_loss_grad
    rng = np.random.default_rng(29)
    ranks = (8, 8, 8)  # shapes the fiber form covers
    coords = draw(rng, dims, 4_000, "uniform")
    vals = rng.standard_normal(4_000).astype(np.float32)
    U = [rng.standard_normal((d, r)).astype(np.float32) for d, r in zip(dims, ranks)]
    G = (rng.standard_normal(ranks) / np.sqrt(np.prod(ranks))).astype(np.float32)
    _, L, dU, dG = gpu_loss_grad(dims, ranks, coords, vals, U, G)
    cc, cv = oracle.coalesce(coords, vals.astype(np.float64))
    Lr, dUr, dGr = oracle.loss_grad(dims, ranks, cc, cv, [u.astype(np.float64) for u in U], G.astype(np.float64))
    assert L == pytest.approx(Lr, rel=1e-4)
    assert rel_fro(dG, dGr) <= 1e-4
    for n in range(3):
        assert rel_fro(dU[n], dUr[n]) <= 1e-4, f"mode {n}"


@pytest.mark.parametrize("mid", [1, 2], ids=["middle-mode2", "middle-mode3"])
def test_mode1_middle_level_against_the_size_guess(mid, monkeypatch):
    """Mode 1's copy is first ordered with its smaller remaining mode as the middle level; when
    the other remaining mode has far fewer distinct (i_1, i_m) pairs the copy is re-sorted from
    that mode's copy.  Here the dimensions point one way and the pairs the other."""
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", "1")
    rng = np.random.default_rng(31 + mid)
    nnz = 40_003
    i1 = rng.integers(0, 100, nnz)
    if mid == 2:  # mode 3 (dim 50) repeats per i_1, mode 2 (dim 40) is the smaller one
        dims = (100, 40, 50)
        coords = np.stack([i1, rng.integers(0, 40, nnz), (i1 * 7 + rng.integers(0, 2, nnz)) % 50])
    else:  # mode 2 (dim 50) repeats per i_1, mode 3 (dim 40) is the smaller one
        dims = (100, 50, 40)
        coords = np.stack([i1, (i1 * 3 + rng.integers(0, 2, nnz)) % 50, rng.integers(0, 40, nnz)])
    coords = coords.astype(np.uint32)
    ranks = (8, 8, 8)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    from tests.gpu_util import lib
    info = lib().tucker_mode_info(ctx, 0)
    assert info["fibers_on"] == 1 and info["fiber_mid_mode"] == mid
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        assert rel_fro(Ys[n], ref[n]) <= TOL, f"mode {n}"
