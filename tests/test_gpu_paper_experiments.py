"""The paper's own experiments that its text fixes, on the GPU against the FP64 oracle.

Fig. 7 (Section IV-C): whole decompositions of 200 x 200 x 200 random tensors with ranks
16 at several sparsities (the figure's points are not printed; two grid points here).
Every unfolding is fat (P = 256 > I = 200), so every mode runs the Gram branch of
Section III-D.  The fit after every sweep within 1e-6; the core, sign-fixed, within 1e-4.

Table III (Section IV-A): the core TTM of a 32 x 32 x I3 tensor with a 32 x I3 factor, as
the core step of a HOOI sweep on a fully listed 32 x 32 x I3 tensor with ranks 32 (QRP
with k = 32 reflectors on 32 x 32 and I3 x I3 Gram matrices).  The fit of every sweep
within 1e-6; the core against the oracle's wherever every pivot decision of the sweep is
separated by more than 1e-8 (modes 1 and 2 keep all 32 directions, so their factors are
bases of R^32 whose column order only a pivot decision fixes); its Frobenius norm, which
no choice of basis changes, always within 1e-6 relative (FP32 TTMc).  I3 = 64 and 256:
at I3 = 32 every factor keeps its whole space, G holds all of X, and the fit is the square
root of a difference at the rounding level of the FP32 Y (no fixed bar on it there)."""
import os

import numpy as np
import pytest

from paper_2010_10638_gb300 import synth
from tests.golden.make_hooi_goldens import oracle_sweeps
from tests.gpu_util import lib, rel_fro, torch
from tests.hooi_canon import canonical

pytestmark = pytest.mark.gpu


def gpu_hooi(inst, iters):
    T = lib()
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(inst.vals).cuda(), w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0])
    try:
        fits = [T.hooi_iter(ctx) for _ in range(iters)]
        U = [T.tucker_get_factor(ctx, n).cpu().numpy() for n in range(len(w.dims))]
        G = T.core_tensor(ctx).cpu().numpy()
    finally:
        T.tucker_free(ctx)
    return fits, U, G


@pytest.mark.parametrize("index", [1, 4], ids=lambda i: f"sparsity-{synth.FIG7_DENSITIES[i]:g}")
def test_fig7_sparsity_point_matches_oracle(index):
    inst = synth.make(synth.fig7_workload(index))
    w = inst.workload
    assert all(r * r > d for r, d in zip(w.ranks, w.dims))  # P_n = 256 > I_n = 200: the Gram branch
    fits, U, G = gpu_hooi(inst, w.iters)
    rec, Uo, Go = oracle_sweeps(inst, threads=os.cpu_count() or 1)
    assert min(min(g) for g in rec["min_gap"]) > 1e-8
    np.testing.assert_allclose(fits, rec["fits"], rtol=0, atol=1e-6)
    Uc, Gc = canonical(U, G)
    Uoc, Goc = canonical(Uo, Go)
    assert rel_fro(Gc, Goc) <= 1e-4
    for n in range(3):
        assert float(np.max(np.abs(Uc[n] - Uoc[n]))) <= 1e-4


@pytest.mark.parametrize("index", [1, 3], ids=lambda i: f"I3-{synth.TABLE3_I3[i]}")
def test_table3_core_ttm_shape_matches_oracle(index):
    inst = synth.make(synth.table3_workload(index))
    w = inst.workload
    assert inst.coords.shape[1] == int(np.prod(w.dims))  # every entry listed
    iters = 2
    fits, U, G = gpu_hooi(inst, iters)
    rec, Uo, Go = oracle_sweeps(inst, iters=iters, threads=os.cpu_count() or 1)
    np.testing.assert_allclose(fits, rec["fits"], rtol=0, atol=1e-6)
    assert np.linalg.norm(G) == pytest.approx(np.linalg.norm(Go), rel=1e-6)
    for n, u in enumerate(U):
        np.testing.assert_allclose(u.T @ u, np.eye(w.ranks[n]), atol=1e-12)
    if min(rec["min_gap"][-1]) > 1e-8:
        Uc, Gc = canonical(U, G)
        Uoc, Goc = canonical(Uo, Go)
        assert rel_fro(Gc, Goc) <= 1e-4
    # the projector of the third factor (the one Table III multiplies by) in any case
    Pg, Po = U[2] @ U[2].T, Uo[2] @ Uo[2].T
    assert np.linalg.norm(Pg - Po) <= 1e-6 * np.sqrt(w.ranks[2])
