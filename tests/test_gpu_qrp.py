"""GPU parity of the FP64 QR with column pivoting (K-c) against the oracle.

Pivots must be identical wherever the top two trailing column norms are separated
by a relative gap > 1e-10 (the GPU downdates norms, the oracle recomputes them);
Q and diag(R) then agree to 1e-12 (same sign convention: v = a + sign(a_1)||a|| e_1)."""
import numpy as np
import pytest

import oracle
from tests.gpu_util import lib, torch

pytestmark = pytest.mark.gpu


def gpu_qrp(A, k):
    T = lib()
    Q, piv, rd = T.qrp_leading(torch.as_tensor(A).cuda(), k)
    return Q.cpu().numpy(), piv.cpu().numpy(), rd.cpu().numpy()


def min_pivot_gap(A, k):
    """Smallest relative gap between the best and second-best trailing norm over the
    first k pivot decisions of exact-norm QRP (computed with the oracle's reflectors)."""
    res = oracle.qrp(A, k)
    W = A[:, res.piv].copy()
    gaps = []
    rest = [c for c in range(A.shape[1]) if c not in set(res.piv.tolist())]
    cols = np.concatenate([res.piv, rest]).astype(int)
    W = A[:, cols]
    Q = res.Q
    for j in range(k):
        R = W - Q[:, :j] @ (Q[:, :j].T @ W)
        nrm = np.sort(np.linalg.norm(R[:, j:], axis=0))[::-1]
        if len(nrm) > 1 and nrm[0] > 0:
            gaps.append((nrm[0] - nrm[1]) / nrm[0])
    return min(gaps) if gaps else 1.0


@pytest.mark.parametrize("m,n,k", [(500, 64, 16), (3000, 256, 16), (64, 64, 64), (257, 33, 8), (40, 300, 20),
                                   (1, 5, 1), (6, 1, 1), (1000, 256, 16), (20_000, 256, 16), (9_001, 130, 12)])
def test_qrp_matches_oracle(m, n, k, qrp_form):
    rng = np.random.default_rng(m * 1000 + n + k)
    A = rng.standard_normal((m, n)) * rng.uniform(0.2, 5.0, n)
    Q, piv, rd = gpu_qrp(A, k)
    ref = oracle.qrp(A, k)
    assert min_pivot_gap(A, k) > 1e-10
    np.testing.assert_array_equal(piv, ref.piv)
    np.testing.assert_allclose(rd, ref.rdiag, rtol=1e-11, atol=1e-12 * abs(ref.rdiag[0]))
    np.testing.assert_allclose(Q, ref.Q, atol=1e-11)
    np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-13)


def test_qrp_rank_deficient_and_zero_columns(qrp_form):
    rng = np.random.default_rng(3)
    A = rng.standard_normal((200, 3)) @ rng.standard_normal((3, 40))
    A[:, 5] = 0.0
    Q, piv, rd = gpu_qrp(A, 6)
    assert np.all(np.isfinite(Q)) and np.all(np.isfinite(rd))
    np.testing.assert_allclose(Q.T @ Q, np.eye(6), atol=1e-12)
    assert np.all(np.abs(rd[3:]) < 1e-10 * abs(rd[0]))
    ref = oracle.qrp(A, 3)
    np.testing.assert_array_equal(piv[:3], ref.piv)
    # the leading 3 columns span the column space
    np.testing.assert_allclose(Q[:, :3] @ (Q[:, :3].T @ A), A, atol=1e-9 * np.abs(A).max())


def test_qrp_all_zero_matrix(qrp_form):
    Q, piv, rd = gpu_qrp(np.zeros((30, 7)), 4)
    np.testing.assert_array_equal(rd, 0.0)
    np.testing.assert_allclose(Q, np.eye(30)[:, :4], atol=0)
    np.testing.assert_array_equal(piv, [0, 1, 2, 3])


def test_qrp_rejects_bad_sizes():
    T = lib()
    with pytest.raises(T.TuckerError):
        T.qrp_leading(torch.zeros((3, 5), dtype=torch.float64, device="cuda"), 4)
    with pytest.raises(T.TuckerError):
        T.qrp_leading(torch.zeros((3, 5), dtype=torch.float64, device="cuda"), 2,
                      work=torch.empty(64, dtype=torch.uint8, device="cuda"))


def test_qrp_runs_as_one_launch(qrp_form):
    """Factorisations with n <= 8192 run as one launch in either single-launch form (the
    multi-kernel form, kept for wider matrices, launches 3k + 3 kernels)."""
    if qrp_form == "multi":
        pytest.skip("the multi-kernel form launches 3k + 3 kernels by design")
    T = lib()
    rng = np.random.default_rng(5)
    for m, n, k in [(50_000, 256, 16), (1000, 256, 16), (40, 6, 4)]:
        A = torch.as_tensor(rng.standard_normal((m, n))).cuda()
        T.qrp_leading(A, k)  # warm-up (first-use attribute set-up)
        torch.cuda.synchronize()
        before = T.tucker_kernel_launches()
        T.qrp_leading(A, k)
        torch.cuda.synchronize()
        assert T.tucker_kernel_launches() - before == 1, (m, n, k)


def test_qrp_cluster_form_on_a_tall_unfolding():
    """50,000 x 256, k = 16 (the shape of a 20M-nonzero tensor's large-mode unfolding):
    several clusters, rows partly in shared memory; the two forms pick the same pivots
    and agree on Q and R to rounding."""
    rng = np.random.default_rng(50)
    A = rng.standard_normal((50_000, 256)) * rng.uniform(0.2, 5.0, 256)
    ref = oracle.qrp(A, 16)
    assert min_pivot_gap(A, 16) > 1e-10
    Q, piv, rd = gpu_qrp(A, 16)
    np.testing.assert_array_equal(piv, ref.piv)
    np.testing.assert_allclose(rd, ref.rdiag, rtol=1e-11)
    np.testing.assert_allclose(Q, ref.Q, atol=1e-11)


def test_multi_kernel_form_on_a_wide_matrix(monkeypatch):
    """The multi-kernel form (3k + 3 launches) on a matrix wider than the persistent
    form's 8192-column limit, forced, against the oracle; and its launch count."""
    monkeypatch.setenv("TUCKER_QRP_FORM", "multi")
    T = lib()
    rng = np.random.default_rng(77)
    m, n, k = 300, 10_000, 8
    A = rng.standard_normal((m, n)) * rng.uniform(0.2, 5.0, n)
    ref = oracle.qrp(A, k)
    assert min_pivot_gap(A, k) > 1e-10
    Ad = torch.as_tensor(A).cuda()
    T.qrp_leading(Ad, k)
    torch.cuda.synchronize()
    before = T.tucker_kernel_launches()
    Q, piv, rd = T.qrp_leading(Ad, k)
    torch.cuda.synchronize()
    assert T.tucker_kernel_launches() - before == 3 * k + 3
    np.testing.assert_array_equal(piv.cpu().numpy(), ref.piv)
    np.testing.assert_allclose(rd.cpu().numpy(), ref.rdiag, rtol=1e-11)
    np.testing.assert_allclose(Q.cpu().numpy(), ref.Q, atol=1e-11)
