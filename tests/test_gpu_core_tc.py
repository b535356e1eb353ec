"""The opt-in core tensor on the tensor cores (TUCKER_CORE_TC=1: tcgen05 kind::f16, every
FP32 input split exactly into three BF16 pieces, six products, FP32 accumulation in tensor
memory over 16 rows, then FP64; Section III-B, eq. core_unfolded: G_(N) = U_N^T Y_(N))
against the FP64 oracle's core of the same Y_(N) and U_N (the GPU's own TTMc output and
FP32 factor copy), and against the default FP64 SIMT form of the same sweep.

Bar: relative Frobenius error 2e-6 on G (FP32-class: the dropped products are about 2^-23
of a product and the tensor-memory accumulation rounds in FP32), fits within 1e-7."""
import os

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import f32_round, lib, rel_fro, torch

pytestmark = pytest.mark.gpu

SHAPES = [  # dims, ranks, nnz: the last mode's P = prod of the other ranks, R_N its rank
    ((300, 200, 1000), (16, 16, 16), 60_000),   # P = 256, R = 16, I_N = 1000
    ((120, 80, 50), (8, 8, 8), 20_000),         # P = 64, R = 8 (N padded to 16)
    ((64, 60, 3000), (10, 10, 32), 80_000),     # P = 100 (not a multiple of 128), R = 32
    ((40, 40, 40, 500), (8, 8, 8, 8), 40_000),  # order 4: P = 512, I_N = 500
    ((100, 90, 70), (12, 5, 48), 30_000),       # R = 48 (N = 48), P = 60
    ((100, 90, 80), (8, 8, 64), 30_000),        # R = 64 (N = 64, 16-row chunks)
    ((50, 40, 5), (6, 7, 5), 800),              # I_N = 5 < one chunk
]


@pytest.mark.parametrize("dims,ranks,nnz", SHAPES, ids=[f"P{np.prod(r[:-1])}-R{r[-1]}-I{d[-1]}" for d, r, _ in SHAPES])
def test_tensor_core_core_matches_oracle(dims, ranks, nnz, monkeypatch):
    T = lib()
    wl = synth.Workload("core-tc", dims, nnz, ranks, 1, 1 + sum(dims), (("uniform",),) * len(dims), "normal")
    w = synth.make(wl)
    N = len(dims)
    ctx = T.tucker_init(dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(),
                        ranks, [torch.as_tensor(u).cuda() for u in w.U0], direct=True)
    try:
        monkeypatch.setenv("TUCKER_CORE_TC", "1")
        fit_tc = T.hooi_iter(ctx)
        G_tc = T.core_tensor(ctx).cpu().numpy()
        # the same step from the same Y_(N) and U_N: the FP64 oracle and the FP64 SIMT form
        Y = T.ttmc_mode(ctx, N - 1).cpu().numpy().astype(np.float64)
        U = T.tucker_get_factor(ctx, N - 1).cpu().numpy()
        G_ref = oracle.core(Y, f32_round([U])[0], ranks)
        err = rel_fro(G_tc, G_ref)
        assert err <= 2e-6, f"core: relative error {err:.2e}"
    finally:
        T.tucker_free(ctx)
    # the default FP64 SIMT form of the whole sweep: same fit to the accuracy of the core
    monkeypatch.delenv("TUCKER_CORE_TC", raising=False)
    ctx = T.tucker_init(dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(),
                        ranks, [torch.as_tensor(u).cuda() for u in w.U0], direct=True)
    try:
        fit64 = T.hooi_iter(ctx)
        G64 = T.core_tensor(ctx).cpu().numpy()
    finally:
        T.tucker_free(ctx)
    assert rel_fro(G_tc, G64) <= 2e-6
    assert abs(fit_tc - fit64) <= 1e-7
