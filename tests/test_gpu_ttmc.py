"""GPU parity of the sparse TTMc (K-b) and the reordering behind it (K-a) against the
FP64 oracle, on identical factor inputs (the FP32 copies the kernel reads).

Tolerance: relative Frobenius error <= 1e-5 on Y_(n) for FP32 factors (the bar stated
for the FP32 form); every element within 1e-5 * max|Y| as well."""
import zlib

import numpy as np
import pytest

import oracle
from paper_2010_10638_gb300 import synth
from tests.gpu_util import f32_round, lib, rel_fro, torch

pytestmark = pytest.mark.gpu

TOL = 1e-5


def run_ttmc_all_modes(dims, ranks, coords, vals, U, bf16=False, **kw):
    T = lib()
    ctx = T.tucker_init(dims, torch.as_tensor(coords.astype(np.int32)).cuda(),
                        torch.as_tensor(vals.astype(np.float32)).cuda(), ranks,
                        [torch.as_tensor(u).cuda() for u in U], bf16=bf16, **kw)
    Ys = [T.ttmc_mode(ctx, n).cpu().numpy() for n in range(len(dims))]
    torch.cuda.synchronize()
    return ctx, Ys


def oracle_all_modes(dims, ranks, coords, vals, U):
    cc, cv = oracle.coalesce(coords, vals.astype(np.float64))
    Uf = f32_round(U)
    return [oracle.ttmc(dims, ranks, cc, cv, n, Uf) for n in range(len(dims))]


CASES = [
    # (name, dims, ranks, nnz, coord recipe)  -- each spans several work units and a ragged tail
    ("order3-r16-uniform", (300, 250, 40), (16, 16, 16), 70_003, "uniform"),
    ("order3-r16-zipf", (2000, 1500, 900), (16, 16, 16), 60_001, "zipf"),
    ("order3-r8", (100, 100, 100), (8, 8, 8), 10_000, "distinct"),
    ("order4-r8", (300, 200, 120, 50), (8, 8, 8, 8), 40_007, "uniform"),
    ("order2-r16", (500, 700), (16, 16), 20_011, "uniform"),
    ("order3-mixed", (200, 300, 150), (8, 16, 16), 30_001, "uniform"),
    ("order3-generic-r10", (200, 180, 160), (10, 10, 10), 25_013, "uniform"),
    ("order5-generic", (20, 18, 16, 14, 12), (3, 4, 2, 3, 2), 9_001, "uniform"),
    ("order3-long-slices", (5, 3000, 2000), (4, 16, 16), 50_000, "uniform"),
    ("order8-generic", (9, 8, 7, 6, 5, 5, 4, 4), (2, 2, 2, 2, 2, 1, 2, 1), 12_007, "uniform"),
]


def draw(rng, dims, nnz, recipe):
    if recipe == "distinct":
        flat = rng.choice(int(np.prod(dims)), size=nnz, replace=False)
        return np.stack(np.unravel_index(flat, dims)).astype(np.uint32)
    out = []
    for d in dims:
        if recipe == "zipf":
            out.append(synth.zipf_indices(rng, d, nnz, 1.2))
        else:
            out.append(rng.integers(0, d, nnz).astype(np.uint32))
    return np.stack(out)


@pytest.mark.parametrize("name,dims,ranks,nnz,recipe", CASES, ids=[c[0] for c in CASES])
def test_ttmc_matches_oracle(name, dims, ranks, nnz, recipe):
    rng = np.random.default_rng(zlib.crc32(name.encode()))
    coords = draw(rng, dims, nnz, recipe)
    vals = rng.standard_normal(nnz).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(len(dims)):
        err = rel_fro(Ys[n], ref[n])
        assert err <= TOL, f"mode {n}: relative Frobenius error {err:.3e}"
        np.testing.assert_allclose(Ys[n], ref[n], rtol=0, atol=TOL * np.abs(ref[n]).max())


def test_ttmc_table1_exact(golden_dir):
    from tests.test_oracle_ttmc import load_table1
    coo, ys = load_table1(golden_dir)
    coords = np.array([[c[m] - 1 for c in coo] for m in range(4)], dtype=np.uint32)
    vals = np.array([c[4] for c in coo], dtype=np.float32)
    U = [np.stack([np.ones(5), np.arange(1, 6)], axis=1).astype(np.float64) for _ in range(4)]
    _, Ys = run_ttmc_all_modes((5, 5, 5, 5), (2, 2, 2, 2), coords, vals, U)
    for n in range(4):
        expected = np.zeros((5, 8))
        for m, row, v in ys:
            if m == n:
                expected[row] = v
        np.testing.assert_array_equal(Ys[n], expected)


def test_ttmc_is_deterministic():
    T = lib()
    w = synth.make("zipf-10k^3", nnz=200_000)
    ctx = T.tucker_init(w.workload.dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(w.vals).cuda(), w.workload.ranks, [torch.as_tensor(u).cuda() for u in w.U0])
    for n in range(3):
        a = T.ttmc_mode(ctx, n).clone()
        b = T.ttmc_mode(ctx, n).clone()
        assert torch.equal(a, b)


def test_empty_tensor_and_empty_rows():
    T = lib()
    dims, ranks = (7, 9, 5), (2, 4, 4)
    U = synth.random_factors(np.random.default_rng(0), dims, ranks)
    ctx = T.tucker_init(dims, torch.zeros((3, 0), dtype=torch.int32, device="cuda"),
                        torch.zeros(0, dtype=torch.float32, device="cuda"), ranks,
                        [torch.as_tensor(u).cuda() for u in U])
    assert T.tucker_nnz(ctx) == 0
    for n in range(3):
        Y = torch.full((dims[n], ctx.P(n)), 7.0, device="cuda")
        T.ttmc_mode(ctx, n, Y)
        assert torch.count_nonzero(Y).item() == 0
    # one nonzero: every other row must be written as zero
    coords = np.array([[3], [8], [0]], dtype=np.uint32)
    vals = np.array([2.5], dtype=np.float32)
    _, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        np.testing.assert_allclose(Ys[n], ref[n], rtol=1e-6, atol=1e-7)


def test_duplicates_are_summed():
    T = lib()
    rng = np.random.default_rng(4)
    dims, ranks = (50, 40, 30), (8, 8, 8)
    base = np.stack([rng.integers(0, d, 3000) for d in dims]).astype(np.uint32)
    coords = np.concatenate([base, base[:, :1000], base[:, :10]], axis=1)
    vals = rng.random(coords.shape[1]).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    cc, cv = oracle.coalesce(coords, vals.astype(np.float64))
    assert T.tucker_nnz(ctx) == cc.shape[1]
    assert T.tucker_norm2(ctx) == pytest.approx(oracle.norm2(cv), rel=1e-12)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        assert rel_fro(Ys[n], ref[n]) <= TOL


def test_invalid_inputs_are_rejected():
    T = lib()
    dims, ranks = (10, 10, 10), (2, 2, 2)
    coords = torch.tensor([[1, 2], [3, 10], [0, 0]], dtype=torch.int32, device="cuda")  # 10 >= dim
    vals = torch.ones(2, device="cuda")
    with pytest.raises(T.TuckerError) as e:
        T.tucker_init(dims, coords, vals, ranks)
    assert e.value.name == "TUCKER_EINVAL"
    coords = torch.tensor([[1, 2], [3, 4], [0, 0]], dtype=torch.int32, device="cuda")
    with pytest.raises(T.TuckerError):
        T.tucker_init(dims, coords, torch.tensor([1.0, float("nan")], device="cuda"), ranks)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_init(dims, coords, vals, (2, 11, 2))
    assert e.value.name == "TUCKER_ERANK"


def test_host_input_path_matches_device_path():
    T = lib()
    w = synth.make("tiny-100^3")
    dims, ranks = w.workload.dims, w.workload.ranks
    c1 = T.tucker_init(dims, w.coords, w.vals, ranks, w.U0)  # host numpy
    c2 = T.tucker_init(dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(), torch.as_tensor(w.vals).cuda(), ranks,
                       [torch.as_tensor(u).cuda() for u in w.U0])
    for n in range(3):
        assert torch.equal(T.ttmc_mode(c1, n), T.ttmc_mode(c2, n))


def test_allocation_failure_is_reported_and_recoverable(monkeypatch):
    T = lib()
    w = synth.make("tiny-100^3")
    dims, ranks = w.workload.dims, w.workload.ranks
    for k in (1, 5, 17):
        monkeypatch.setenv("TUCKER_FAIL_ALLOC_AT", str(k))
        with pytest.raises(T.TuckerError) as e:
            T.tucker_init(dims, w.coords, w.vals, ranks, w.U0)
        assert e.value.name == "TUCKER_ENOMEM"
    monkeypatch.delenv("TUCKER_FAIL_ALLOC_AT")
    ctx = T.tucker_init(dims, w.coords, w.vals, ranks, w.U0)
    assert T.tucker_nnz(ctx) == w.workload.nnz


def test_bounded_wait_times_out_and_context_survives():
    """A device wait that can never finish gives up after its poll limit, the timeout is
    reported by the next synchronising call, and the context keeps working."""
    T = lib()
    w = synth.make("tiny-100^3")
    ctx = T.tucker_init(w.workload.dims, w.coords, w.vals, w.workload.ranks, w.U0)
    T.tucker_sync_status(ctx)  # clean
    T.tucker_selftest_wait(ctx, 20_000)
    with pytest.raises(T.TuckerError) as e:
        T.tucker_sync_status(ctx)
    assert e.value.name == "TUCKER_ETIMEOUT"
    T.tucker_sync_status(ctx)  # cleared
    Y = T.ttmc_mode(ctx, 0)
    assert torch.isfinite(Y).all()
    assert 0.0 < T.hooi_iter(ctx) < 1.0


@pytest.mark.parametrize("dims", [(3, 1 << 17, 7), (5, (1 << 24) + 3, 2), (1, 40, 30), (20, 1, 1)],
                         ids=["17-bit", "25-bit", "one-row-mode1", "one-row-modes23"])
def test_sort_key_widths(dims):
    """Indices of 17 and 25 bits (three and four sort passes of under 8 bits each) and
    modes with a single index (no pass): the mode copies, hence Y, against the oracle."""
    rng = np.random.default_rng(sum(dims))
    nnz = 30_011
    coords = np.stack([rng.integers(0, d, nnz) for d in dims]).astype(np.uint32)
    vals = rng.standard_normal(nnz).astype(np.float32)
    ranks = tuple(min(2, d) for d in dims)
    U = synth.random_factors(rng, dims, ranks)
    _, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        assert rel_fro(Ys[n], ref[n]) <= TOL, f"mode {n}"


def test_duplicate_groups_across_warp_and_tile_edges():
    """Groups of equal coordinates that straddle 32-position steps, 512-position warps and
    8192-position tiles of the coalescing pass (one group of 20,000 copies), summed in FP64."""
    T = lib()
    rng = np.random.default_rng(41)
    dims, ranks = (64, 48, 40), (4, 4, 4)
    base = np.stack([rng.integers(0, d, 30_000) for d in dims]).astype(np.uint32)
    reps = rng.integers(1, 70, base.shape[1])
    coords = np.repeat(base, reps, axis=1)
    big = np.repeat(np.array([[5], [7], [9]], dtype=np.uint32), 20_000, axis=1)
    coords = np.concatenate([coords, big], axis=1)
    perm = rng.permutation(coords.shape[1])
    coords = coords[:, perm]
    vals = rng.standard_normal(coords.shape[1]).astype(np.float32)
    U = synth.random_factors(rng, dims, ranks)
    ctx, Ys = run_ttmc_all_modes(dims, ranks, coords, vals, U)
    cc, cv = oracle.coalesce(coords, vals.astype(np.float64))
    assert T.tucker_nnz(ctx) == cc.shape[1]
    assert T.tucker_norm2(ctx) == pytest.approx(oracle.norm2(cv), rel=1e-12)
    ref = oracle_all_modes(dims, ranks, coords, vals, U)
    for n in range(3):
        assert rel_fro(Ys[n], ref[n]) <= TOL, f"mode {n}"


def test_lib_setup():
    T = lib()
    T.tucker_lib_setup()
    T.tucker_lib_setup()  # again: no effect
    with pytest.raises(T.TuckerError) as e:
        T.tucker_lib_setup(torch.cuda.device_count() + 3)
    assert e.value.name == "TUCKER_ECUDA"
    assert torch.cuda.current_device() == 0
    w = synth.make("tiny-100^3")
    ctx = T.tucker_init(w.workload.dims, w.coords, w.vals, w.workload.ranks, w.U0)
    assert T.tucker_nnz(ctx) == w.workload.nnz


def test_sort_lookback_wait_is_bounded():
    """A sort pass whose look-back waits for counts that never come gives up after its
    poll limit, reports TUCKER_ETIMEOUT, stores nothing, and the device stays usable."""
    T = lib()
    assert T.tucker_selftest_sort_wait(20_000) == "TUCKER_ETIMEOUT"
    with pytest.raises(T.TuckerError):
        T.tucker_selftest_sort_wait(0)
    w = synth.make("tiny-100^3")
    ctx = T.tucker_init(w.workload.dims, w.coords, w.vals, w.workload.ranks, w.U0)
    assert T.tucker_nnz(ctx) == w.workload.nnz
    assert 0.0 < T.hooi_iter(ctx) < 1.0
