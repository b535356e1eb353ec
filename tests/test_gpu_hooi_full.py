"""GPU HOOI (Algorithm 2) at the workload recipes' full sizes and sweep counts, against
the FP64 oracle: zipf-10k^3 (1M nonzeros, 10 sweeps) run live, order4-5M (5M, 10 sweeps,
FP32 and BF16 factors) and skew-20M (20M, 10 sweeps) against stored oracle results
(tests/golden/hooi_<name>.json, written by tests/golden/make_hooi_goldens.py, which
calls only the oracle).

Bars (FP32 TTMc): the fit after every sweep within 1e-6 (absolute); the core of the last
sweep, sign-fixed (tests/hooi_canon.py), within 1e-4 relative Frobenius; every factor's
sketch U_n^T W_n within 1e-4 absolute (an error of the factor's columns of about that
size; W_n has unit-variance entries) on the columns the QRP determines (|r_jj| >= 1e-3
|r_11| in the oracle's last sweep).  The stored results record the smallest gap
between the top two trailing column norms of every pivot decision; all of them are far
above the FP32 rounding of Y_(n) (smallest 7.6e-6 relative), so the same pivots must be
chosen and the factors compared column by column.

BF16 factors (order4-5M, skew-20M): the fit after every sweep within 1e-2 of the FP64
oracle's (the BF16 form's stated 1e-2 bar, taken on the fit); the observed error is printed."""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch
from tests.hooi_canon import canonical, sketch

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
FIT_TOL, G_TOL, SKETCH_TOL, BF16_FIT_TOL = 1e-6, 1e-4, 1e-4, 1e-2


def gpu_run(inst, bf16=False):
    T = lib()
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0],
                        bf16=bf16)
    try:
        fits = [T.hooi_iter(ctx) for _ in range(w.iters)]
        U = [T.tucker_get_factor(ctx, n).cpu().numpy() for n in range(len(w.dims))]
        G = T.core_tensor(ctx).cpu().numpy()
        nnz, nx2 = T.tucker_nnz(ctx), T.tucker_norm2(ctx)
    finally:
        T.tucker_free(ctx)
    return fits, U, G, nnz, nx2


def check_model(U, G, G_ref_canon, sketches_ref, ranks, rdiag_last):
    """Core and factors of the last sweep.  A factor column j is compared only where the
    oracle's QRP determined it: |r_jj| >= 1e-3 |r_11|.  Below that the column is a
    direction of (numerically) zero weight in Y_(n) (order4-5M's last mode ends with
    |r_88| = 2e-21 |r_11|), which any rounding may turn; the core's entries along it are
    at the same level, so the core comparison needs no such mask."""
    for n, u in enumerate(U):
        np.testing.assert_allclose(u.T @ u, np.eye(ranks[n]), atol=1e-12)
    Uc, Gc = canonical(U, G)
    err_g = rel_fro(Gc, G_ref_canon)
    assert err_g <= G_TOL, f"core: relative error {err_g:.2e}"
    for n in range(len(U)):
        rd = np.abs(np.asarray(rdiag_last[n]))
        keep = rd >= 1e-3 * rd[0]
        assert keep[0]
        d = float(np.max(np.abs(sketch(Uc[n], n) - np.asarray(sketches_ref[n]))[keep]))
        assert d <= SKETCH_TOL, f"factor {n}: sketch differs by {d:.2e} ({int(keep.sum())} determined columns)"
    return err_g


def test_zipf_1M_ten_sweeps_live_against_oracle():
    inst = synth.make("zipf-10k^3")
    w = inst.workload
    fits, U, G, _, _ = gpu_run(inst)
    ref = oracle.hooi(w.dims, w.ranks, inst.coords, inst.vals.astype(np.float64), inst.U0, w.iters,
                      threads=os.cpu_count() or 1)
    np.testing.assert_allclose(fits, ref.fits, rtol=0, atol=FIT_TOL)
    Uo, Go = canonical(ref.U, ref.G)
    check_model(U, G, Go, [sketch(Uo[n], n) for n in range(3)], w.ranks, ref.rdiags[-1])


@pytest.mark.parametrize("name", ["order4-5M", "skew-20M"])
def test_full_config_ten_sweeps_against_stored_oracle(name):
    with open(os.path.join(GOLDEN, f"hooi_{name}.json")) as f:
        ref = json.load(f)
    inst = synth.make(name)
    w = inst.workload
    assert ref["sweeps"] == w.iters and tuple(ref["ranks"]) == tuple(w.ranks) and ref["seed"] == w.seed
    assert min(min(g) for g in ref["min_gap"]) > 1e-6  # every pivot decision well separated
    fits, U, G, nnz, nx2 = gpu_run(inst)
    assert nnz == ref["nnz_coalesced"]
    assert nx2 == pytest.approx(ref["normX2"], rel=1e-12)
    np.testing.assert_allclose(fits, ref["fits"], rtol=0, atol=FIT_TOL)
    check_model(U, G, np.asarray(ref["G_canon"]).reshape(w.ranks), ref["sketch"], w.ranks, ref["rdiag"][-1])


@pytest.mark.parametrize("name", ["order4-5M", "skew-20M"])
def test_bf16_factors_ten_sweeps_against_stored_oracle(name):
    with open(os.path.join(GOLDEN, f"hooi_{name}.json")) as f:
        ref = json.load(f)
    fits, U, _, _, _ = gpu_run(synth.make(name), bf16=True)
    err = np.abs(np.asarray(fits) - np.asarray(ref["fits"]))
    print(f"{name} BF16 factors: fit error after each sweep {', '.join(f'{e:.1e}' for e in err)}")
    assert np.all(err <= BF16_FIT_TOL)
    for n, u in enumerate(U):
        np.testing.assert_allclose(u.T @ u, np.eye(u.shape[1]), atol=1e-12)
