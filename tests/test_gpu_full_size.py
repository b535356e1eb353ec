"""Parity of the TTMc (Algorithm 2, Eq. 4) at the workload recipes' full sizes, in the
launch configuration the benchmark times, on sampled rows of Y_(n) that the FP64 oracle
computes from the nonzeros of those rows alone; with the seeded initial factors and again
after three HOOI sweeps (factors from the QRP, FP32-rounded as the kernels read them).

Tolerance: the componentwise bound of a floating-point sum.  Each entry of Y_(n) is a sum
of k_i products, one per nonzero of row i, each product a value times N-1 factor entries;
FP32 rounding of the products and of a sum of k terms in any order leaves
    |Y - Y_exact| <= (k_i + N) u_32 (|X| x_{m != n} |U_m|^T)
with u_32 = 2^-24 and the absolute-value contraction on the right.  This is the bound that
holds whatever the conditioning: after sweeps on a tensor of structureless random values
(fit near 0) HOOI turns the factors toward a few heavy indices and some rows of Y cancel
almost exactly, so an error relative to |Y| itself has no fixed bar there.  The BF16-factor
form adds one BF16 rounding (u_16 = 2^-8) per factor entry and per partial product, (N+1)
per term."""
import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import f32_round, lib, torch

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U16 = 2.0 ** -8
ROWS = 48


def sampled_rows(inst, mode, rng):
    present = np.unique(inst.coords[mode])
    pick = np.sort(rng.choice(present, size=min(ROWS, present.size), replace=False))
    sel = np.isin(inst.coords[mode], pick)
    return pick, np.ascontiguousarray(inst.coords[:, sel]), inst.vals[sel].astype(np.float64)


def check_modes(T, ctx, inst, U, bf16, rng, label):
    w = inst.workload
    N = len(w.dims)
    Uf = f32_round(U)
    for n in range(N):
        Y = T.ttmc_mode(ctx, n).cpu().numpy().astype(np.float64)
        pick, cc, cv = sampled_rows(inst, n, rng)
        cc, cv = oracle.coalesce(cc, cv)
        ref = oracle.ttmc(w.dims, w.ranks, cc, cv, n, Uf)[pick]
        absref = oracle.ttmc(w.dims, w.ranks, cc, np.abs(cv), n, [np.abs(u) for u in Uf])[pick]
        k = np.bincount(cc[n], minlength=w.dims[n])[pick].astype(np.float64)[:, None]
        per_term = (N + 1) * U16 if bf16 else 0.0
        bound = (per_term + (k + N) * U32) * absref
        d = np.abs(Y[pick] - ref)
        worst = float(np.max(d / np.maximum(bound, 1e-300)))
        assert np.all(d <= bound), f"{label} mode {n}: error reaches {worst:.2f}x the componentwise bound"
        assert np.all(np.isfinite(Y[pick]))


FULL = [("zipf-10k^3", False), ("order4-5M", False), ("order4-5M", True), ("skew-20M", False),
        ("skew-20M", True), ("completion-10M", False)]


@pytest.mark.parametrize("name,bf16", FULL, ids=[f"{n}-{'bf16' if b else 'fp32'}" for n, b in FULL])
def test_full_size_sampled_rows_within_componentwise_bound(name, bf16):
    T = lib()
    inst = synth.make(name)
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0],
                        bf16=bf16)
    rng = np.random.default_rng(17)
    try:
        check_modes(T, ctx, inst, inst.U0, bf16, rng, "initial factors")
        for _ in range(3):
            T.hooi_iter(ctx)
        U = [T.tucker_get_factor(ctx, m).cpu().numpy() for m in range(len(w.dims))]
        check_modes(T, ctx, inst, U, bf16, rng, "after 3 sweeps")
    finally:
        T.tucker_free(ctx)
