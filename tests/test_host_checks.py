"""Host-side argument checks of the C ABI, on the CPU: every call below is refused (or, for
k = 0, completed) before the library touches the GPU, with the status include/tucker.h
states for it."""
import ctypes

import pytest

OK, EINVAL, ERANK = 0, 1, 2


@pytest.fixture(scope="module")
def lib():
    from paper_2010_10638_gb300 import build
    lib = ctypes.CDLL(build.build())
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.tucker_init.argtypes = [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(i64), i64, vp, vp,
                                ctypes.POINTER(ctypes.c_int), vp, ctypes.c_uint64, ctypes.c_uint32, vp]
    lib.qrp_leading.argtypes = [vp, i64, i64, i64, ctypes.c_int, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.qrp_leading_work_bytes.argtypes = [i64, i64, ctypes.c_int]
    lib.qrp_leading_work_bytes.restype = ctypes.c_size_t
    for name in ("ttmc_mode", "hooi_iter", "core_tensor"):
        getattr(lib, name).argtypes = [vp] + ([ctypes.c_int, vp, vp] if name == "ttmc_mode" else [vp, vp])
    lib.ttmc_mode_norms.argtypes = [vp, ctypes.c_int, vp, vp, vp]
    lib.tucker_get_factor.argtypes = [vp, ctypes.c_int, vp, vp]
    return lib


def init(lib, dims, ranks, nnz=0, coords=None, vals=None, out=True):
    n = len(dims)
    d = (ctypes.c_int64 * n)(*dims)
    r = (ctypes.c_int * n)(*ranks)
    h = ctypes.c_void_p()
    return lib.tucker_init(ctypes.byref(h) if out else None, n, d, nnz, coords, vals, r, None, 0, 0, None)


def test_tucker_init_refuses_bad_shapes(lib):
    assert init(lib, (10, 10, 10), (2, 2, 2), out=False) == EINVAL          # no handle to fill
    assert init(lib, (10,), (2,)) == EINVAL                                   # order 1
    assert init(lib, (10,) * 9, (1,) * 9) == EINVAL                           # order above the maximum
    assert init(lib, (10, 0, 10), (2, 1, 2)) == EINVAL                        # an empty dimension
    assert init(lib, (10, 10, 10), (2, 2, 2), nnz=-1) == EINVAL               # negative nonzero count
    assert init(lib, (10, 10, 10), (2, 2, 2), nnz=5) == EINVAL                # nonzeros without coordinates
    assert init(lib, (10, 10, 10), (2, 11, 2)) == ERANK                       # rank above its dimension
    assert init(lib, (100, 100, 100), (65, 2, 2)) == ERANK                    # rank above 64
    assert init(lib, (200, 200, 200, 200), (64, 64, 64, 64)) == ERANK         # prod R above 2^20
    assert init(lib, (10, 10, 10), (0, 2, 2)) == ERANK                        # rank 0


def test_calls_without_a_context_are_refused(lib):
    assert lib.ttmc_mode(None, 0, None, None) == EINVAL
    assert lib.ttmc_mode_norms(None, 0, None, None, None) == EINVAL
    assert lib.hooi_iter(None, None, None) == EINVAL
    assert lib.core_tensor(None, None, None) == EINVAL
    assert lib.tucker_get_factor(None, 0, None, None) == EINVAL


def test_qrp_leading_refuses_bad_sizes(lib):
    buf = ctypes.create_string_buffer(4096 + 256)
    base = ctypes.addressof(buf)
    aligned = ctypes.c_void_p((base + 255) // 256 * 256)
    dummy = ctypes.c_void_p(aligned.value)
    assert lib.qrp_leading(dummy, -1, 4, 4, 1, dummy, None, None, aligned, 4096, None) == EINVAL   # m < 0
    assert lib.qrp_leading(dummy, 8, 4, 3, 1, dummy, None, None, aligned, 4096, None) == EINVAL    # lda < n
    assert lib.qrp_leading(dummy, 8, 4, 4, 5, dummy, None, None, aligned, 4096, None) == ERANK     # k > n
    assert lib.qrp_leading(dummy, 3, 4, 4, 4, dummy, None, None, aligned, 4096, None) == ERANK     # k > m
    assert lib.qrp_leading(dummy, 100, 100, 100, 65, dummy, None, None, aligned, 4096, None) == ERANK  # k > 64
    assert lib.qrp_leading(None, 8, 4, 4, 0, None, None, None, None, 0, None) == OK                # k = 0: nothing to do
    assert lib.qrp_leading(None, 8, 4, 4, 2, dummy, None, None, aligned, 4096, None) == EINVAL     # no A
    misaligned = ctypes.c_void_p(aligned.value + 8)
    assert lib.qrp_leading(dummy, 8, 4, 4, 2, dummy, None, None, misaligned, 4096, None) == EINVAL  # work not 256-aligned
    assert lib.qrp_leading(dummy, 8, 4, 4, 2, dummy, None, None, aligned, 16, None) == EINVAL       # work too small


def test_qrp_work_bytes_grow_with_the_problem(lib):
    small = lib.qrp_leading_work_bytes(1000, 64, 8)
    assert small > 0
    assert lib.qrp_leading_work_bytes(50_000, 256, 16) > small
    assert lib.qrp_leading_work_bytes(1000, 64, 16) >= small
