"""The BF16-factor form of the TTMc (factors stored in BF16, tensor-core products,
FP32 accumulation) against the FP64 oracle: relative Frobenius error <= 1e-2 on
Y_(n), the bar stated for the BF16 form; and the opt-in TMA-fed BF16 form against the
register-staged one (bit for bit)."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch

pytestmark = pytest.mark.gpu

CASES = [("order3-r16-zipf", (3000, 2000, 800), (16, 16, 16), 120_000),
         ("order4-r8", (400, 300, 200, 60), (8, 8, 8, 8), 80_000),
         ("order3-r16x8", (500, 400, 300), (16, 16, 8), 50_000)]


def bf16_round(a):
    t = torch.as_tensor(np.asarray(a, dtype=np.float32)).to(torch.bfloat16).to(torch.float64)
    return t.numpy()


@pytest.mark.parametrize("name,dims,ranks,nnz", CASES, ids=[c[0] for c in CASES])
def test_bf16_form_within_1e2(name, dims, ranks, nnz):
    T = lib()
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    coords = np.stack([synth.zipf_indices(rng, d, nnz, 1.1) if "zipf" in name else rng.integers(0, d, nnz)
                       for d in dims]).astype(np.uint32)
    vals = rng.lognormal(0.0, 1.0, nnz).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx = T.tucker_init(dims, torch.as_tensor(coords.astype(np.int32)).cuda(), torch.as_tensor(vals).cuda(), ranks,
                        [torch.as_tensor(u).cuda() for u in U], bf16=True)
    cc, cv = oracle.coalesce(coords, vals.astype(np.float64))
    Ub = [bf16_round(u) for u in U]
    Uf = [u.astype(np.float32).astype(np.float64) for u in U]
    for n in range(len(dims)):
        Y = T.ttmc_mode(ctx, n).cpu().numpy()
        err_b = rel_fro(Y, oracle.ttmc(dims, ranks, cc, cv, n, Ub))
        err_f = rel_fro(Y, oracle.ttmc(dims, ranks, cc, cv, n, Uf))
        assert err_b <= 1e-2, f"mode {n}: {err_b:.3e} vs BF16-rounded factors"
        assert err_f <= 1e-2, f"mode {n}: {err_f:.3e} vs FP32 factors"


@pytest.mark.parametrize("name,nnz", [("zipf-10k^3", 200_000), ("skew-20M", 300_000)])
def test_tma_fed_bf16_form_equals_register_staged_form(name, nnz, monkeypatch):
    """The opt-in BF16 form whose factor rows arrive by TMA row gathers (gather4 into a
    4-stage shared-memory ring, mbarrier completion) computes the same products in the
    same order as the register-staged BF16 form: Y equal bit for bit on every mode."""
    T = lib()
    w = synth.make(name, nnz=nnz)
    ctx = T.tucker_init(w.workload.dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(w.vals).cuda(), w.workload.ranks, [torch.as_tensor(u).cuda() for u in w.U0],
                        bf16=True)
    for n in range(3):
        monkeypatch.setenv("TUCKER_TTMC_TMA", "0")
        Y0 = T.ttmc_mode(ctx, n).clone()
        monkeypatch.setenv("TUCKER_TTMC_TMA", "1")
        Y1 = T.ttmc_mode(ctx, n).clone()
        torch.cuda.synchronize()
        T.tucker_sync_status(ctx)  # no bounded wait gave up
        assert torch.equal(Y0, Y1), f"mode {n}"
    T.tucker_free(ctx)
