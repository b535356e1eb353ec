"""The split-TF32 tensor-core form of the FP32 TTMc (opt-in, TUCKER_TTMC_TF32=1; left rank
16, last rank 16 or 8) against the FP64 oracle, on identical FP32 factor inputs.

Each FP32 operand is split into two TF32 parts and three products are summed; the
dropped terms are below 2^-21 of |A||B| per product, so the bar is the FP32 form's:
relative Frobenius error <= 1e-5 and every element within 1e-5 * max|Y|.  Covered: the
nonzero and fiber forms, slices split over work units (32-nonzero units), mixed ranks
(modes the form does not cover run the SIMT form), determinism, and HOOI fits within
1e-6 of the oracle."""
import os
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch
from tests.test_gpu_ttmc import draw, oracle_all_modes, run_ttmc_all_modes

pytestmark = pytest.mark.gpu

TOL = 1e-5

CASES = [
    # (name, dims, ranks, nnz, coord recipe)
    ("r16-uniform", (300, 250, 40), (16, 16, 16), 70_003, "uniform"),
    ("r16-zipf", (2000, 1500, 900), (16, 16, 16), 60_001, "zipf"),
    ("r16-r8", (80, 16, 300), (16, 16, 8), 25_003, "uniform"),
    ("mixed", (200, 300, 150), (8, 16, 16), 30_001, "uniform"),
    ("long-slices", (5, 3000, 2000), (4, 16, 16), 50_000, "uniform"),
    ("long-fibers", (60, 16, 500), (16, 16, 16), 40_009, "uniform"),
    ("dense-ish", (30, 30, 30), (16, 16, 16), 20_000, "distinct"),
]


@pytest.fixture
def tf32(monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_TF32", "1")


@pytest.mark.parametrize("fibers", ["1", "0"], ids=["fibers", "nonzeros"])
@pytest.mark.parametrize("chunk", [None, "32"], ids=["default-units", "small-units"])
@pytest.mark.parametrize("name,dims,ranks,nnz,recipe", CASES, ids=[c[0] for c in CASES])
def test_tf32_form_matches_oracle(name, dims, ranks, nnz, recipe, chunk, fibers, tf32, monkeypatch):
    monkeypatch.setenv("TUCKER_TTMC_FIBERS", fibers)
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


def test_tf32_form_is_deterministic(tf32):
    T = lib()
    w = synth.make("zipf-10k^3", nnz=200_000)
    ctx = T.tucker_init(w.workload.dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(w.vals).cuda(), w.workload.ranks, [torch.as_tensor(u).cuda() for u in w.U0])
    for n in range(3):
        a = T.ttmc_mode(ctx, n).clone()
        b = T.ttmc_mode(ctx, n).clone()
        assert torch.equal(a, b)


def test_tf32_hooi_matches_oracle(tf32):
    T = lib()
    wl = synth.Workload("skew-small", (3000, 3000, 200), 400_000, (16, 16, 16), 3, 91,
                        (("zipf", 1.2), ("uniform",), ("uniform",)), "lognormal")
    w = synth.make(wl)
    ctx = T.tucker_init(wl.dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(),
                        wl.ranks, [torch.as_tensor(u).cuda() for u in w.U0])
    fits = [T.hooi_iter(ctx) for _ in range(3)]
    ref = oracle.hooi(wl.dims, wl.ranks, w.coords, w.vals.astype(np.float64), w.U0, 3, threads=os.cpu_count() or 1)
    np.testing.assert_allclose(fits, ref.fits, rtol=0, atol=1e-6)
