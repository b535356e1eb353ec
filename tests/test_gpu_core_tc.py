"""The core tensor on the tensor cores (core_tc_kernel: tcgen05 kind::f16; Section III-B,
eq. core_unfolded: G_(N) = U_N^T Y_(N)) against the FP64 oracle's core of the same Y_(N) and
U_N (the GPU's own TTMc output and FP64 factor), and against the FP64 SIMT form of the same
sweep (TUCKER_CORE_TC=0).

The tensor-core form splits Y's columns and U's columns into four 8-bit fixed-point slices
against a shared power of two per column and row range; every tensor-memory accumulation is
an exact integer sum.  Its only errors are the parts of Y and U below the last slice
(under 2^-33 of the column's largest entry; for an entry of G at most sqrt(I_N) 2^-32 of the
largest entry of its Y column) and FP64 additions.  Bars: relative Frobenius error 1e-8 on G,
fits within 1e-8 of the FP64 form."""
import os

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch

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
        G_ref = oracle.core(Y, U, ranks)
        err = rel_fro(G_tc, G_ref)
        assert err <= 1e-8, f"core: relative error {err:.2e}"
    finally:
        T.tucker_free(ctx)
    # the FP64 SIMT form of the whole sweep: same fit to the accuracy of the core
    monkeypatch.setenv("TUCKER_CORE_TC", "0")
    ctx = T.tucker_init(dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(),
                        ranks, [torch.as_tensor(u).cuda() for u in w.U0], direct=True)
    try:
        fit64 = T.hooi_iter(ctx)
        G64 = T.core_tensor(ctx).cpu().numpy()
    finally:
        T.tucker_free(ctx)
    assert rel_fro(G_tc, G64) <= 1e-8
    assert abs(fit_tc - fit64) <= 1e-8
