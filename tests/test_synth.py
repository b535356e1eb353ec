"""The seeded input generators follow the recipes they state (scaled-down draws): Zipf
rank frequencies against the analytic law, uniform modes, value distributions, the
completion recipe's noise level, orthonormal initial factors, determinism."""
import numpy as np
import pytest

from paper_2010_10638_gb300 import synth


def zipf_pmf(n, s):
    w = np.arange(1, n + 1, dtype=np.float64) ** (-s)
    return w / w.sum()


@pytest.mark.parametrize("n,s", [(1000, 1.2), (10_000, 1.1)])
def test_zipf_rank_frequencies_follow_the_law(n, s):
    rng = np.random.default_rng(3)
    size = 400_000
    idx = synth.zipf_indices(rng, n, size, s)
    assert idx.min() >= 0 and idx.max() < n
    counts = np.sort(np.bincount(idx, minlength=n))[::-1].astype(np.float64)
    pmf = zipf_pmf(n, s)
    # the heaviest ranks: within 4 standard deviations of the binomial counts
    for r in range(5):
        mean = size * pmf[r]
        assert abs(counts[r] - mean) <= 4 * np.sqrt(mean * (1 - pmf[r])), (r, counts[r], mean)
    # the slope of log frequency against log rank over ranks 1..50 is -s
    r = np.arange(1, 51)
    slope = np.polyfit(np.log(r), np.log(counts[:50]), 1)[0]
    assert abs(slope + s) < 0.05


def test_skew_recipe_modes_and_values():
    inst = synth.make("skew-20M", nnz=300_000)
    w = inst.workload
    assert w.dims == (50_000, 50_000, 1_000) and w.ranks == (16, 16, 16)
    c = inst.coords
    assert c.shape == (3, 300_000) and c.dtype == np.uint32
    for m in range(3):
        assert c[m].max() < w.dims[m]
    # mode 1 Zipf(1.2): the heaviest index holds about P(rank 1) of the nonzeros
    top = np.bincount(c[0]).max() / c.shape[1]
    assert abs(top - zipf_pmf(w.dims[0], 1.2)[0]) < 0.01
    # mode 3 uniform over 1,000 indices: counts close to 300 each
    cnt = np.bincount(c[2], minlength=1000)
    assert abs(cnt.mean() - 300) < 1e-9 and cnt.std() < 1.3 * np.sqrt(300)
    # lognormal(0, 1) values
    lv = np.log(inst.vals.astype(np.float64))
    assert abs(lv.mean()) < 0.01 and abs(lv.std() - 1.0) < 0.01


def test_completion_recipe_is_a_tucker_model_plus_noise():
    inst = synth.make("completion-10M", nnz=50_000)
    w = inst.workload
    G, U = inst.model["G"], inst.model["U"]
    c = inst.coords
    clean = np.einsum("abc,za,zb,zc->z", G, U[0][c[0]], U[1][c[1]], U[2][c[2]])
    noise = inst.vals.astype(np.float64) - clean
    assert abs(noise.std() / w.noise_sigma - 1.0) < 0.05
    assert np.linalg.norm(clean) > 10 * np.linalg.norm(noise)


def test_initial_factors_are_orthonormal_and_draws_are_seeded():
    a = synth.make("tiny-100^3")
    b = synth.make("tiny-100^3")
    for u, r in zip(a.U0, a.workload.ranks):
        np.testing.assert_allclose(u.T @ u, np.eye(r), atol=1e-12)
    np.testing.assert_array_equal(a.coords, b.coords)
    np.testing.assert_array_equal(a.vals, b.vals)
    c = synth.make("tiny-100^3", seed=5)
    assert not np.array_equal(a.coords, c.coords)
