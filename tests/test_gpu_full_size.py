"""Parity of the TTMc (Algorithm 2, inner loop; Section III-C) at the workload recipes'
full sizes, in the launch configuration the benchmark times, on sampled rows of Y_(n)
that the FP64 oracle computes from those rows' nonzeros alone: 48 rows drawn uniformly
from the non-empty rows plus the 8 heaviest rows of every mode (on skew-20M the heaviest
mode-1 row holds about 4M nonzeros and runs through the split-slice path and its fixup
kernel); with the seeded initial factors and again after three HOOI sweeps (factors from
the QRP, FP32-rounded as the kernels read them).

Two bars.
1. The stated accuracy target of each form: relative Frobenius error over the sampled rows
   <= 1e-5 (FP32 factors) or 1e-2 (BF16 factors), with the initial factors.
2. Componentwise, with any factors: the error bound of a floating-point sum whose terms
   are products of N factors, evaluated in a tree of depth D:
       |Y - Y_exact| <= (D + N) u_32 (|X| x_{m != n} |U_m|^T)
   (u_32 = 2^-24, the absolute-value contraction on the right), with D the depth of the
   summation the kernels actually perform for that row, read from the mode's layout
   (tucker_mode_info):
     nonzero form: the lanes of a group add every NG-th nonzero of a work unit in order
       (at most min(k_i, chunk) terms), 5 shuffle levels merge the groups, and a row split
       over p pieces adds them in the fixup kernel (ceil(p/8) + 8 additions);
     fiber form: a fiber's sum t_f adds its at most fiber_cap nonzeros in order, the update
       adds at most min(k_i, fchunk) fiber terms per unit plus 5 shuffle levels, and the
       fixup as above over the fiber pieces.
   This holds whatever the conditioning: after sweeps on a tensor of structureless random
   values (fit near 0) some sampled rows cancel almost exactly, and an error relative to
   |Y| itself has no fixed bar there.  The BF16-factor form adds one BF16 rounding
   (u_16 = 2^-8) per factor entry and per partial product, (N + 1) per term."""
import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import f32_round, lib, rel_fro, torch

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
U16 = 2.0 ** -8
ROWS, HEAVY = 48, 8
TARGET_BAR = {False: 1e-5, True: 1e-2}  # relative Frobenius: FP32 / BF16 factors


def sampled_rows(inst, mode, rng):
    counts = np.bincount(inst.coords[mode], minlength=inst.workload.dims[mode])
    present = np.flatnonzero(counts)
    heavy = np.argsort(counts, kind="stable")[::-1][:HEAVY]
    pick = np.union1d(rng.choice(present, size=min(ROWS, present.size), replace=False), heavy[counts[heavy] > 0])
    sel = np.isin(inst.coords[mode], pick)
    return pick, np.ascontiguousarray(inst.coords[:, sel]), inst.vals[sel].astype(np.float64)


def summation_depth(info, k, bf16):
    """Additions on the longest path from a term to Y(i, :) for rows with k nonzeros (the
    BF16-factor form always runs the nonzero form)."""
    def fixup(pieces):
        return np.where(pieces > 1, np.ceil(pieces / 8.0) + 8, 0)
    if info["fibers_on"] and not bf16:
        fc = info["fchunk"]
        return info["fiber_cap"] + np.minimum(k, fc) + 5 + fixup(np.ceil(k / fc))
    c = info["chunk"]
    return np.minimum(k, c) + 5 + fixup(np.ceil(k / c))


def check_modes(T, ctx, inst, U, bf16, rng, label, target_bar):
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
        D = summation_depth(T.tucker_mode_info(ctx, n), k, bf16)
        per_term = (N + 1) * U16 if bf16 else 0.0
        bound = (per_term + (D + N) * U32) * absref
        d = np.abs(Y[pick] - ref)
        worst = float(np.max(d / np.maximum(bound, 1e-300)))
        assert np.all(d <= bound), f"{label} mode {n}: error reaches {worst:.2f}x the componentwise bound"
        assert np.all(np.isfinite(Y[pick]))
        if target_bar:
            err = rel_fro(Y[pick], ref)
            assert err <= TARGET_BAR[bf16], f"{label} mode {n}: relative Frobenius error {err:.2e}"
        print(f"{w.name} {'bf16' if bf16 else 'fp32'} {label} mode {n}: {pick.size} rows, heaviest "
              f"{int(k.max())} nonzeros, worst {worst:.3f} of the bound, rel. Frobenius {rel_fro(Y[pick], ref):.2e}")


FULL = [("zipf-10k^3", False), ("order4-5M", False), ("order4-5M", True), ("skew-20M", False),
        ("skew-20M", True), ("completion-10M", False)]


@pytest.mark.parametrize("name,bf16", FULL, ids=[f"{n}-{'bf16' if b else 'fp32'}" for n, b in FULL])
def test_full_size_sampled_rows_against_oracle(name, bf16):
    T = lib()
    inst = synth.make(name)
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0],
                        bf16=bf16)
    rng = np.random.default_rng(17)
    try:
        check_modes(T, ctx, inst, inst.U0, bf16, rng, "initial factors", target_bar=True)
        for _ in range(3):
            T.hooi_iter(ctx)
        U = [T.tucker_get_factor(ctx, m).cpu().numpy() for m in range(len(w.dims))]
        check_modes(T, ctx, inst, U, bf16, rng, "after 3 sweeps", target_bar=False)
    finally:
        T.tucker_free(ctx)


def test_full_size_zipf_every_row_against_oracle():
    """zipf-10k^3 (1M nonzeros) whole: every row of every mode's Y against the oracle,
    relative Frobenius <= 1e-5 with the initial factors."""
    T = lib()
    inst = synth.make("zipf-10k^3")
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0])
    cc, cv = oracle.coalesce(inst.coords, inst.vals.astype(np.float64))
    try:
        for n in range(3):
            Y = T.ttmc_mode(ctx, n).cpu().numpy().astype(np.float64)
            ref = oracle.ttmc(w.dims, w.ranks, cc, cv, n, f32_round(inst.U0))
            assert rel_fro(Y, ref) <= 1e-5, f"mode {n}: {rel_fro(Y, ref):.2e}"
    finally:
        T.tucker_free(ctx)
