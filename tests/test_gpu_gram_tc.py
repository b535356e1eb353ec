"""The Gram matrix S = Y_(n) Y_(n)^T of fat unfoldings (Section III-D: P_n > I_n, the QRP
factors S) on the tensor cores (gram_tc_kernel: exact 8-bit fixed-point slices per row of Y
over blocks of 128 columns), against the FP64 SIMT form of the same sweeps
(TUCKER_CORE_TC=0 runs both the Gram matrix and the core in FP64).

Both forms compute S to FP64 rounding except for the parts of Y below the last slice (under
2^-33 of a row's largest entry in a block), so the sweeps agree: fits within 1e-9, and the
factors' projectors within 1e-7 (the QRP of the Gram matrix amplifies an S difference by the
conditioning of its leading block).  One case has a 1,100-row Gram matrix, above the
tensor-core form's 1,024 rows: it runs the FP64 form in both settings (equal bit for bit)."""
import numpy as np
import pytest

from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, torch

pytestmark = pytest.mark.gpu

CASES = [  # dims, ranks, nnz: every listed mode has P_n > I_n
    ((200, 200, 200), (16, 16, 16), 40_000),         # Fig. 7 shape: m = 200, n = 256
    ((64, 60, 1000), (32, 32, 20), 60_000),          # m = 64, 60 (n = 640), m = 1000 (n = 1024)
    ((30, 40, 50, 60), (8, 8, 8, 8), 30_000),        # order 4: n = 512
    ((64, 40, 1100), (64, 32, 8), 40_000),           # mode 3: m = 1100 > 1024 (FP64 form)
]


def sweeps(T, inst, iters):
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(), torch.as_tensor(inst.vals).cuda(),
                        w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0])
    try:
        fits = [T.hooi_iter(ctx) for _ in range(iters)]
        U = [T.tucker_get_factor(ctx, n).cpu().numpy() for n in range(len(w.dims))]
    finally:
        T.tucker_free(ctx)
    return np.array(fits), U


@pytest.mark.parametrize("dims,ranks,nnz", CASES, ids=[f"{'x'.join(map(str, d))}-R{r[-1]}" for d, r, _ in CASES])
def test_tensor_core_gram_matches_fp64_form(dims, ranks, nnz, monkeypatch):
    T = lib()
    wl = synth.Workload("gram-tc", dims, nnz, ranks, 1, 7 + sum(dims), (("uniform",),) * len(dims), "normal")
    inst = synth.make(wl)
    assert all(int(np.prod([r for m, r in enumerate(ranks) if m != n])) > d for n, d in enumerate(dims))
    monkeypatch.delenv("TUCKER_CORE_TC", raising=False)
    f_tc, U_tc = sweeps(T, inst, 3)
    monkeypatch.setenv("TUCKER_CORE_TC", "0")
    f_64, U_64 = sweeps(T, inst, 3)
    np.testing.assert_allclose(f_tc, f_64, rtol=0, atol=1e-9)
    for n in range(len(dims)):
        d = np.linalg.norm(U_tc[n] @ U_tc[n].T - U_64[n] @ U_64[n].T)
        assert d <= 1e-7, f"mode {n}: projector difference {d:.2e}"
