"""qrp_leading_noalloc: the QRP entry point for callers that cannot allocate device
memory (its scratch is a fixed device array inside the library).  Checked through
the C ABI against qrp_leading, which takes caller-provided scratch, on two calls in a
row: the second call reuses the array the first one left dirty.

This file is collected last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import ctypes

import numpy as np
import pytest

from tests.gpu_util import lib, torch

pytestmark = pytest.mark.gpu


def _call_noalloc(L, A, k):
    m, n = A.shape
    Q = torch.full((m, k), float("nan"), dtype=torch.float64, device="cuda")
    piv = torch.full((k,), -1, dtype=torch.int64, device="cuda")
    rd = torch.full((k,), float("nan"), dtype=torch.float64, device="cuda")
    rc = L.qrp_leading_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, n, k, ctypes.c_void_p(Q.data_ptr()),
                               ctypes.c_void_p(piv.data_ptr()), ctypes.c_void_p(rd.data_ptr()),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, f"qrp_leading_noalloc returned {rc}"
    torch.cuda.synchronize()
    return Q.cpu().numpy(), piv.cpu().numpy(), rd.cpu().numpy()


def _call_with_work(L, A, k):
    m, n = A.shape
    need = L.qrp_leading_work_bytes(m, n, k)
    work = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    Q = torch.empty((m, k), dtype=torch.float64, device="cuda")
    piv = torch.empty(k, dtype=torch.int64, device="cuda")
    rd = torch.empty(k, dtype=torch.float64, device="cuda")
    rc = L.qrp_leading(ctypes.c_void_p(A.data_ptr()), m, n, n, k, ctypes.c_void_p(Q.data_ptr()),
                       ctypes.c_void_p(piv.data_ptr()), ctypes.c_void_p(rd.data_ptr()),
                       ctypes.c_void_p(work.data_ptr()), work.numel(),
                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0
    assert L.qrp_leading_sync_status(ctypes.c_void_p(work.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    torch.cuda.synchronize()
    return Q.cpu().numpy(), piv.cpu().numpy(), rd.cpu().numpy()


def test_noalloc_matches_qrp_leading_on_two_calls_in_a_row():
    T = lib()
    L = T.load()
    rng = np.random.default_rng(2024)
    # a larger problem first, then smaller ones that run on the scratch left behind; k = 48
    # is beyond the cluster form (k <= 32) and runs the persistent form on the same array
    for m, n, k in [(4000, 256, 16), (300, 40, 12), (3000, 128, 48)]:
        A = torch.as_tensor(rng.standard_normal((m, n)) * rng.uniform(0.2, 5.0, n)).cuda()
        assert L.qrp_leading_work_bytes(m, n, k) <= L.qrp_leading_noalloc_max_bytes()
        Q, piv, rd = _call_noalloc(L, A, k)
        assert L.qrp_leading_noalloc_sync_status(ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        Qr, pivr, rdr = _call_with_work(L, A, k)
        np.testing.assert_array_equal(piv, pivr)
        np.testing.assert_allclose(rd, rdr, rtol=1e-11, atol=1e-12 * abs(rdr[0]))
        np.testing.assert_allclose(Q, Qr, atol=1e-11)
        np.testing.assert_allclose(Q.T @ Q, np.eye(k), atol=1e-13)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    T = lib()
    L = T.load()
    cap = L.qrp_leading_noalloc_max_bytes()
    m, n, k = 2_000_000, 64, 16  # V alone is m * k * 8 = 256 MB
    assert L.qrp_leading_work_bytes(m, n, k) > cap
    # buffers of the full size, so that the call stays in bounds even if it did not refuse
    A = torch.zeros((m, n), dtype=torch.float64, device="cuda")
    Q = torch.empty((m, k), dtype=torch.float64, device="cuda")
    rc = L.qrp_leading_noalloc(ctypes.c_void_p(A.data_ptr()), m, n, n, k, ctypes.c_void_p(Q.data_ptr()), None, None,
                               None)
    torch.cuda.synchronize()
    assert T.STATUS[rc] == "TUCKER_EINVAL"
