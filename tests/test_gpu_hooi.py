"""GPU HOOI (Algorithm 2: TTMc -> QRP per mode, then the core and the fit) against the
FP64 oracle: the fit after every sweep within 1e-6, the factors' subspaces and the
core tensor close, pivot choices identical."""
import os

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch
from tests.hooi_canon import canonical

pytestmark = pytest.mark.gpu


def gpu_hooi(dims, ranks, coords, vals, U0, iters, **kw):
    T = lib()
    ctx = T.tucker_init(dims, torch.as_tensor(coords.astype(np.int32)).cuda(), torch.as_tensor(vals).cuda(), ranks,
                        [torch.as_tensor(u).cuda() for u in U0], **kw)
    fits = [T.hooi_iter(ctx) for _ in range(iters)]
    U = [T.tucker_get_factor(ctx, n).cpu().numpy() for n in range(len(dims))]
    G = T.core_tensor(ctx).cpu().numpy()
    return ctx, fits, U, G


def check_against_oracle(w, iters, fit_tol=1e-6, **kw):
    dims, ranks = w.workload.dims, w.workload.ranks
    ctx, fits, U, G = gpu_hooi(dims, ranks, w.coords, w.vals, w.U0, iters, **kw)
    ref = oracle.hooi(dims, ranks, w.coords, w.vals.astype(np.float64), w.U0, iters,
                      direct=kw.get("direct", False), threads=os.cpu_count() or 1)
    np.testing.assert_allclose(fits, ref.fits, rtol=0, atol=fit_tol)
    for n in range(len(dims)):
        np.testing.assert_allclose(U[n].T @ U[n], np.eye(ranks[n]), atol=1e-12)
        Pg, Po = U[n] @ U[n].T, ref.U[n] @ ref.U[n].T
        assert np.linalg.norm(Pg - Po) <= 1e-4 * np.sqrt(ranks[n])
    # the core itself (Section III-B), with every factor column's sign fixed on both sides
    Uc, Gc = canonical(U, G)
    Uo, Go = canonical(ref.U, ref.G)
    assert rel_fro(Gc, Go) <= 1e-4, f"core: relative error {rel_fro(Gc, Go):.2e}"
    for n in range(len(dims)):
        assert float(np.max(np.abs(Uc[n] - Uo[n]))) <= 1e-4
    return fits, ref


def test_hooi_tiny_config_matches_oracle(qrp_form):
    w = synth.make("tiny-100^3")
    fits, ref = check_against_oracle(w, w.workload.iters)
    assert all(0.0 <= f <= 1.0 for f in fits)


def test_hooi_order4_fat_mode_gram_and_direct(qrp_form):
    # last mode 40 < P = 8*8*8 = 512: the paper's Gram branch; direct QRP as a flag
    rng = np.random.default_rng(2)
    wl = synth.Workload("order4-small", (300, 250, 200, 40), 60_000, (8, 8, 8, 8), 3, 77, (("uniform",),) * 4,
                        "normal")
    w = synth.make(wl)
    check_against_oracle(w, 3)
    check_against_oracle(w, 3, direct=True)


def test_hooi_exact_low_rank_recovery():
    rng = np.random.default_rng(12)
    dims, ranks = (40, 30, 20), (4, 3, 2)
    X, coords, vals = synth.low_rank_dense(rng, dims, ranks)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    ctx, fits, U, G = gpu_hooi(dims, ranks, coords, vals.astype(np.float32), U0, 2)
    # FP32 values and FP32 TTMc: ||X||^2 - ||G||^2 ~ 1e-7 ||X||^2 under a square root
    assert fits[-1] > 1.0 - 3e-3
    Xh = G
    for m in range(3):
        Xh = np.moveaxis(np.tensordot(Xh, U[m], axes=([m], [1])), -1, m)
    assert np.linalg.norm(Xh - X) / np.linalg.norm(X) < 1e-5


def test_hooi_zipf_small_matches_oracle(qrp_form):
    w = synth.make("zipf-10k^3", nnz=100_000)
    check_against_oracle(w, 2)


def test_hooi_skew_recipe_small_matches_oracle(qrp_form):
    # the 50,000 x 50,000 x 1,000 shape at 300k nonzeros: FP32 unfoldings of 50,000 x 256
    w = synth.make("skew-20M", nnz=300_000)
    check_against_oracle(w, 2)


def test_core_tensor_requires_a_sweep():
    T = lib()
    w = synth.make("tiny-100^3")
    ctx = T.tucker_init(w.workload.dims, w.coords, w.vals, w.workload.ranks, w.U0)
    with pytest.raises(T.TuckerError) as e:
        T.core_tensor(ctx)
    assert e.value.name == "TUCKER_ESTATE"


def test_seeded_initial_factors_are_orthonormal():
    T = lib()
    w = synth.make("tiny-100^3")
    ctx = T.tucker_init(w.workload.dims, w.coords, w.vals, w.workload.ranks, None, seed=5)
    for n in range(3):
        U = T.tucker_get_factor(ctx, n).cpu().numpy()
        np.testing.assert_allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-13)
    f = T.hooi_iter(ctx)
    assert 0.0 < f < 1.0


def test_hooi_rejects_ranks_qrp_cannot_produce():
    # order 2, ranks (6, 8): mode 2 would need 8 QRP columns from a 80 x 6 unfolding
    T = lib()
    rng = np.random.default_rng(0)
    dims, ranks = (90, 80), (6, 8)
    coords = np.stack([rng.integers(0, d, 500) for d in dims]).astype(np.uint32)
    vals = rng.random(500).astype(np.float32)
    U0 = [synth.orthonormal_factor(rng, d, r) for d, r in zip(dims, ranks)]
    ctx = T.tucker_init(dims, coords, vals, ranks, U0)  # allowed: the loss/adjoint works with any ranks
    with pytest.raises(T.TuckerError) as e:
        T.hooi_iter(ctx)
    assert e.value.name == "TUCKER_ERANK"
