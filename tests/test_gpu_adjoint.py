"""GPU adjoint (tucker_loss_grad, K-e) against the FP64 oracle's loss and gradients,
which are themselves pinned by finite differences (tests/test_oracle_adjoint.py).

Tolerance: relative error <= 1e-4 on the loss, every dU_n and dG (FP32 arithmetic)."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, rel_fro, torch

pytestmark = pytest.mark.gpu
TOL = 1e-4


def distinct_coords(rng, dims, nnz):
    flat = rng.choice(int(np.prod(dims, dtype=np.int64)), size=nnz, replace=False)
    return np.stack(np.unravel_index(flat, dims)).astype(np.uint32)


def gpu_loss_grad(dims, ranks, coords, vals, U, G):
    T = lib()
    ctx = T.tucker_init(dims, torch.as_tensor(coords.astype(np.int32)).cuda(), torch.as_tensor(vals).cuda(), ranks,
                        [torch.as_tensor(u.astype(np.float64)).cuda() for u in U])
    loss, dU, dG = T.tucker_loss_grad(ctx, [torch.as_tensor(u.astype(np.float32)).cuda() for u in U],
                                      torch.as_tensor(G.astype(np.float32)).cuda())
    torch.cuda.synchronize()
    return ctx, float(loss.item()), [d.cpu().numpy() for d in dU], dG.cpu().numpy()


CASES = [("order3-r10", (60, 50, 40), (10, 10, 10), 20_000), ("order3-r8", (80, 70, 60), (8, 8, 8), 30_000),
         ("order3-r16", (60, 64, 70), (16, 16, 16), 15_000), ("order4", (20, 18, 16, 14), (4, 3, 4, 2), 12_000),
         ("order2", (90, 80), (6, 8), 3_000), ("order3-mixed", (40, 50, 30), (3, 8, 5), 10_000)]


@pytest.mark.parametrize("name,dims,ranks,nnz", CASES, ids=[c[0] for c in CASES])
def test_loss_grad_matches_oracle(name, dims, ranks, nnz):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    coords = distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = [rng.standard_normal((d, r)).astype(np.float32) for d, r in zip(dims, ranks)]
    G = (rng.standard_normal(ranks) / np.sqrt(np.prod(ranks))).astype(np.float32)
    _, L, dU, dG = gpu_loss_grad(dims, ranks, coords, vals, U, G)
    Lr, dUr, dGr = oracle.loss_grad(dims, ranks, coords, vals.astype(np.float64),
                                    [u.astype(np.float64) for u in U], G.astype(np.float64))
    assert L == pytest.approx(Lr, rel=TOL)
    assert rel_fro(dG, dGr) <= TOL
    for n in range(len(dims)):
        assert rel_fro(dU[n], dUr[n]) <= TOL, f"mode {n}"


def test_completion_workload_sample_and_multilinear_identity():
    """The completion workload (Tucker-model values + noise) at 100k observed entries:
    parity with the oracle, and <dG, G> = <dU_n, U_n> for every n (each equals
    sum_z e_z xhat_z because xhat is linear in G and in every U_n)."""
    inst = synth.make("completion-10M", nnz=100_000)
    w = inst.workload
    cc, cv = oracle.coalesce(inst.coords, inst.vals.astype(np.float64))
    rng = np.random.default_rng(3)
    U = [(inst.model["U"][m] + 0.1 * rng.standard_normal(inst.model["U"][m].shape)).astype(np.float32)
         for m in range(3)]
    G = inst.model["G"].astype(np.float32)
    _, L, dU, dG = gpu_loss_grad(w.dims, w.ranks, cc, cv.astype(np.float32), U, G)
    Lr, dUr, dGr = oracle.loss_grad(w.dims, w.ranks, cc, cv.astype(np.float32).astype(np.float64),
                                    [u.astype(np.float64) for u in U], G.astype(np.float64))
    assert L == pytest.approx(Lr, rel=TOL)
    assert rel_fro(dG, dGr) <= TOL
    for n in range(3):
        assert rel_fro(dU[n], dUr[n]) <= TOL
    ref = float(np.sum(dG.astype(np.float64) * G))
    for n in range(3):
        assert float(np.sum(dU[n].astype(np.float64) * U[n])) == pytest.approx(ref, rel=1e-4)


def test_completion_10M_finite_differences_on_a_1000_entry_subsample():
    """The completion workload's own check: 1,000 observed entries drawn (seeded) from the
    completion-10M tensor itself, the parameters near the generating model.  The GPU
    gradients (FP32) against central finite differences (h = 1e-6) of the FP64 oracle's
    loss on the same entries, along four random directions over G and every U_m at once,
    and on single entries of G and of factor rows the subsample touches; and against the
    oracle's analytic gradients.  Bars: oracle vs finite differences 1e-6, GPU vs finite
    differences and vs the oracle 1e-4 (relative to the derivative, or to the largest
    entry of that gradient for single entries)."""
    T = lib()
    inst = synth.make("completion-10M")
    w = inst.workload
    rng = np.random.default_rng(55)
    pick = np.sort(rng.choice(w.nnz, size=1000, replace=False))
    coords = np.ascontiguousarray(inst.coords[:, pick])
    vals = inst.vals[pick]
    U = [(inst.model["U"][m] + 0.1 * rng.standard_normal(inst.model["U"][m].shape)).astype(np.float32)
         for m in range(3)]
    G = inst.model["G"].astype(np.float32)
    _, L, dU, dG = gpu_loss_grad(w.dims, w.ranks, coords, vals, U, G)
    U64 = [u.astype(np.float64) for u in U]
    G64 = G.astype(np.float64)
    v64 = vals.astype(np.float64)
    Lr, dUr, dGr = oracle.loss_grad(w.dims, w.ranks, coords, v64, U64, G64)
    assert L == pytest.approx(Lr, rel=TOL)
    assert rel_fro(dG, dGr) <= TOL
    for n in range(3):
        assert rel_fro(dU[n], dUr[n]) <= TOL

    def loss(Us, Gs):
        return oracle.loss_grad(w.dims, w.ranks, coords, v64, Us, Gs)[0]

    h = 1e-6
    for _ in range(4):
        D = [rng.standard_normal(u.shape) for u in U64]
        DG = rng.standard_normal(G64.shape)
        fd = (loss([u + h * d for u, d in zip(U64, D)], G64 + h * DG)
              - loss([u - h * d for u, d in zip(U64, D)], G64 - h * DG)) / (2 * h)
        an_o = sum(float(np.sum(d * g)) for d, g in zip(D, dUr)) + float(np.sum(DG * dGr))
        an_g = sum(float(np.sum(d * g.astype(np.float64))) for d, g in zip(D, dU)) + float(np.sum(DG * dG))
        assert abs(an_o - fd) <= 1e-6 * abs(fd)
        assert abs(an_g - fd) <= TOL * abs(fd)
    # single entries: 8 of the core, 8 of each factor in rows the subsample touches
    for _ in range(8):
        q = tuple(int(rng.integers(0, r)) for r in w.ranks)
        Gp, Gm = G64.copy(), G64.copy()
        Gp[q] += h
        Gm[q] -= h
        fd = (loss(U64, Gp) - loss(U64, Gm)) / (2 * h)
        assert abs(float(dG[q]) - fd) <= TOL * float(np.max(np.abs(dGr)))
        assert abs(float(dGr[q]) - fd) <= 1e-6 * float(np.max(np.abs(dGr)))
    for m in range(3):
        for _ in range(8):
            i = int(coords[m, rng.integers(0, coords.shape[1])])
            r = int(rng.integers(0, w.ranks[m]))
            Up = [u.copy() for u in U64]
            Um = [u.copy() for u in U64]
            Up[m][i, r] += h
            Um[m][i, r] -= h
            fd = (loss(Up, G64) - loss(Um, G64)) / (2 * h)
            assert abs(float(dU[m][i, r]) - fd) <= TOL * float(np.max(np.abs(dUr[m])))
            assert abs(float(dUr[m][i, r]) - fd) <= 1e-6 * float(np.max(np.abs(dUr[m])))


def test_directional_finite_difference_on_gpu():
    T = lib()
    rng = np.random.default_rng(9)
    dims, ranks, nnz = (50, 40, 30), (5, 4, 6), 8_000
    coords = distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = [rng.standard_normal((d, r)).astype(np.float32) for d, r in zip(dims, ranks)]
    G = (rng.standard_normal(ranks) / 10).astype(np.float32)
    ctx, L, dU, dG = gpu_loss_grad(dims, ranks, coords, vals, U, G)
    D = [rng.standard_normal(u.shape).astype(np.float32) for u in U]
    DG = rng.standard_normal(ranks).astype(np.float32)
    h = 1e-3

    def loss_at(s):
        Us = [torch.as_tensor(u + s * d).cuda() for u, d in zip(U, D)]
        Gs = torch.as_tensor(G + s * DG).cuda()
        return float(T.tucker_loss_grad(ctx, Us, Gs)[0].item())

    fd = (loss_at(h) - loss_at(-h)) / (2 * h)
    an = sum(float(np.sum(d.astype(np.float64) * g)) for d, g in zip(D, dU)) + float(np.sum(DG * dG))
    assert fd == pytest.approx(an, rel=2e-3)


def test_autograd_function_and_descent():
    from paper_2010_10638_gb300.autograd import tucker_loss
    T = lib()
    inst = synth.make("completion-10M", nnz=200_000)
    w = inst.workload
    ctx = T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(), torch.as_tensor(inst.vals).cuda(),
                        w.ranks, [torch.as_tensor(u).cuda() for u in inst.U0])
    rng = np.random.default_rng(1)
    U = [torch.tensor(inst.model["U"][m] + 0.3 * rng.standard_normal(inst.model["U"][m].shape), dtype=torch.float32,
                      device="cuda", requires_grad=True) for m in range(3)]
    G = torch.tensor(inst.model["G"], dtype=torch.float32, device="cuda", requires_grad=True)
    loss = tucker_loss(ctx, G, U)
    loss.backward()
    L2, dU, dG = T.tucker_loss_grad(ctx, [u.detach() for u in U], G.detach())
    assert torch.equal(G.grad, dG)
    for u, d in zip(U, dU):
        assert torch.equal(u.grad, d)
    opt = torch.optim.Adam([G, *U], lr=1e-2)
    first = float(loss.item())
    for _ in range(30):
        opt.zero_grad()
        l = tucker_loss(ctx, G, U)
        l.backward()
        opt.step()
    assert float(l.item()) < 0.5 * first


def test_loss_grad_is_deterministic():
    T = lib()
    rng = np.random.default_rng(2)
    dims, ranks, nnz = (200, 150, 100), (8, 8, 8), 50_000
    coords = distinct_coords(rng, dims, nnz)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = [rng.standard_normal((d, r)).astype(np.float32) for d, r in zip(dims, ranks)]
    G = rng.standard_normal(ranks).astype(np.float32)
    ctx, *_ = gpu_loss_grad(dims, ranks, coords, vals, U, G)
    Ut = [torch.as_tensor(u).cuda() for u in U]
    Gt = torch.as_tensor(G).cuda()
    a = T.tucker_loss_grad(ctx, Ut, Gt)
    b = T.tucker_loss_grad(ctx, Ut, Gt)
    assert torch.equal(a[0], b[0]) and torch.equal(a[2], b[2])
    for x, y in zip(a[1], b[1]):
        assert torch.equal(x, y)
