"""Python binding of libtucker (include/tucker.h): argument marshalling only.

Every function here has the name of the C entry point it calls and forwards torch
tensors as raw device pointers together with the current CUDA stream.  There is no
CPU fallback: if the library is not built, or there is no GPU, the calls raise.

    import torch
    from paper_2010_10638_gb300 import tucker as T
    ctx = T.tucker_init(dims, coords, vals, ranks, U0)   # coords: int32 [N, nnz] (cuda or cpu)
    fit = T.hooi_iter(ctx)
    G = T.core_tensor(ctx)
    T.tucker_free(ctx)
"""

from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
# TUCKER_LIB_PATH selects another build of the same library (the checked build of the tests)
LIB_PATH = os.environ.get("TUCKER_LIB_PATH") or os.path.join(_HERE, "_build", "libtucker.so")

TUCKER_F_BF16_FACTORS = 0x1
TUCKER_F_QRP_DIRECT = 0x2
TUCKER_F_HOST_INPUT = 0x4
TUCKER_F_FIT_DEVICE = 0x8
TUCKER_F_UNPIPELINED = 0x20
TUCKER_F_TTMC_NORMS = 0x40

STATUS = {0: "TUCKER_OK", 1: "TUCKER_EINVAL", 2: "TUCKER_ERANK", 3: "TUCKER_ENOMEM", 4: "TUCKER_ECUDA",
          5: "TUCKER_ETIMEOUT", 6: "TUCKER_ESTATE"}

EXPORTS = ["tucker_init", "ttmc_mode", "ttmc_mode_norms", "qrp_leading", "qrp_leading_work_bytes", "hooi_iter", "core_tensor",
           "tucker_get_factor", "tucker_set_factor", "tucker_loss_grad", "tucker_nnz", "tucker_norm2",
           "tucker_sync_status", "tucker_free", "tucker_status_str", "tucker_last_error", "tucker_set_profiling",
           "tucker_phase_times", "tucker_kernel_launches", "qrp_leading_noalloc", "qrp_leading_noalloc_max_bytes",
           "tucker_selftest_wait", "tucker_mode_info", "qrp_leading_sync_status",
           "qrp_leading_noalloc_sync_status", "tucker_fp32_fma_tflops", "tucker_hooi_graph", "tucker_lib_setup",
           "tucker_selftest_sort_wait", "tucker_check_site"]


class TuckerError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{where}: {self.name}" + (f" ({detail})" if detail else ""))


_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libtucker is not built ({path} missing): run `python -m paper_2010_10638_gb300.build`")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, i64, u64, u32, cint, csz, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                         ctypes.c_int, ctypes.c_size_t, ctypes.c_double)
    lib.tucker_init.argtypes = [P(vp), cint, P(i64), i64, vp, vp, P(cint), vp, u64, u32, vp]
    lib.ttmc_mode.argtypes = [vp, cint, vp, vp]
    lib.ttmc_mode_norms.argtypes = [vp, cint, vp, vp, vp]
    lib.qrp_leading.argtypes = [vp, i64, i64, i64, cint, vp, vp, vp, vp, csz, vp]
    lib.qrp_leading_work_bytes.argtypes = [i64, i64, cint]
    lib.qrp_leading_work_bytes.restype = csz
    lib.hooi_iter.argtypes = [vp, vp, vp]
    lib.core_tensor.argtypes = [vp, vp, vp]
    lib.tucker_get_factor.argtypes = [vp, cint, vp, vp]
    lib.tucker_set_factor.argtypes = [vp, cint, vp, vp]
    lib.tucker_loss_grad.argtypes = [vp, P(vp), vp, vp, P(vp), vp, vp]
    lib.tucker_nnz.argtypes = [vp]
    lib.tucker_nnz.restype = i64
    lib.tucker_norm2.argtypes = [vp]
    lib.tucker_norm2.restype = dbl
    lib.tucker_sync_status.argtypes = [vp, vp]
    lib.tucker_free.argtypes = [vp]
    lib.tucker_free.restype = None
    lib.tucker_status_str.argtypes = [cint]
    lib.tucker_status_str.restype = ctypes.c_char_p
    lib.tucker_last_error.argtypes = [vp]
    lib.tucker_last_error.restype = ctypes.c_char_p
    lib.tucker_set_profiling.argtypes = [vp, cint]
    lib.tucker_set_profiling.restype = cint
    lib.tucker_phase_times.argtypes = [vp, P(ctypes.c_float), cint]
    lib.tucker_phase_times.restype = cint
    lib.qrp_leading_noalloc.argtypes = [vp, i64, i64, i64, cint, vp, vp, vp, vp]
    lib.qrp_leading_noalloc.restype = cint
    lib.qrp_leading_noalloc_max_bytes.argtypes = []
    lib.qrp_leading_noalloc_max_bytes.restype = csz
    lib.tucker_selftest_wait.argtypes = [vp, u64, vp]
    lib.tucker_selftest_wait.restype = cint
    lib.qrp_leading_sync_status.argtypes = [vp, vp]
    lib.qrp_leading_sync_status.restype = cint
    lib.qrp_leading_noalloc_sync_status.argtypes = [vp]
    lib.qrp_leading_noalloc_sync_status.restype = cint
    lib.tucker_hooi_graph.argtypes = [vp, cint, vp, vp]
    lib.tucker_hooi_graph.restype = cint
    lib.tucker_fp32_fma_tflops.argtypes = [cint, vp]
    lib.tucker_fp32_fma_tflops.restype = dbl
    lib.tucker_mode_info.argtypes = [vp, cint, P(i64), cint]
    lib.tucker_mode_info.restype = cint
    lib.tucker_selftest_sort_wait.argtypes = [u64, vp]
    lib.tucker_selftest_sort_wait.restype = cint
    lib.tucker_lib_setup.argtypes = [cint]
    lib.tucker_lib_setup.restype = cint
    lib.tucker_check_site.argtypes = []
    lib.tucker_check_site.restype = ctypes.c_int32
    lib.tucker_kernel_launches.argtypes = []
    lib.tucker_kernel_launches.restype = ctypes.c_uint64
    for name in ("tucker_init", "ttmc_mode", "qrp_leading", "hooi_iter", "core_tensor", "tucker_get_factor",
                 "tucker_set_factor", "tucker_loss_grad", "tucker_sync_status"):
        getattr(lib, name).restype = cint
    _lib = lib
    return lib


def _stream(stream=None) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _check(rc: int, where: str, ctx=None):
    if rc != 0:
        detail = ""
        if ctx is not None and getattr(ctx, "handle", None):
            detail = load().tucker_last_error(ctx.handle).decode()
        raise TuckerError(rc, where, detail)


def _dev(t: torch.Tensor, dtype, what: str) -> torch.Tensor:
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what}: expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{what}: expected dtype {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{what}: expected a contiguous tensor")
    return t


class Context:
    """Owns one tucker_ctx handle; keeps the metadata needed to size outputs."""

    def __init__(self, handle, dims, ranks, flags):
        self.handle = handle
        self.dims = tuple(int(d) for d in dims)
        self.ranks = tuple(int(r) for r in ranks)
        self.flags = flags
        self.N = len(self.dims)

    def P(self, mode: int) -> int:
        return int(np.prod([r for m, r in enumerate(self.ranks) if m != mode], dtype=np.int64))

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                load().tucker_free(self.handle)
            except Exception:
                pass
            self.handle = None


# --------------------------------------------------------------------------- entry points
def tucker_lib_setup(device: int | None = None) -> None:
    """One-time set-up of the library on a device (memory pool, first allocation, the
    initialisation's kernels); optional, otherwise done on first use."""
    lib = load()
    dev = torch.cuda.current_device() if device is None else int(device)
    _check(lib.tucker_lib_setup(dev), "tucker_lib_setup")


def tucker_init(dims, coords, vals, ranks, U0=None, seed: int = 0, bf16: bool = False, direct: bool = False,
                fit_device: bool = False, unpipelined: bool = False, ttmc_norms: bool = False,
                stream=None) -> Context:
    """coords: int32/uint32 [N, nnz]; vals: float32 [nnz]; U0: list of N float64 [I_m, R_m] or None.
    CUDA tensors are passed as device pointers; CPU tensors / numpy arrays as host pointers
    (TUCKER_F_HOST_INPUT; all inputs must then be on the host)."""
    lib = load()
    N = len(dims)
    flags = (TUCKER_F_BF16_FACTORS if bf16 else 0) | (TUCKER_F_QRP_DIRECT if direct else 0) | (
        TUCKER_F_FIT_DEVICE if fit_device else 0) | (
        TUCKER_F_UNPIPELINED if unpipelined else 0) | (TUCKER_F_TTMC_NORMS if ttmc_norms else 0)
    on_host = not (isinstance(coords, torch.Tensor) and coords.is_cuda)
    keep = []
    if on_host:
        flags |= TUCKER_F_HOST_INPUT
        c = torch.as_tensor(np.ascontiguousarray(np.asarray(coords).astype(np.uint32).view(np.int32)))
        v = torch.as_tensor(np.ascontiguousarray(np.asarray(vals, dtype=np.float32)))
        if U0 is not None:
            u = torch.as_tensor(np.concatenate([np.ascontiguousarray(np.asarray(x, dtype=np.float64)).reshape(-1)
                                                for x in U0]))
        keep += [c, v]
    else:
        c = coords if coords.dtype == torch.int32 else coords.to(torch.int32)
        c = _dev(c.contiguous(), torch.int32, "coords")
        v = _dev(vals.contiguous(), torch.float32, "vals")
        if U0 is not None:  # one buffer, filled by device-to-device copies
            parts = [_dev(x.contiguous(), torch.float64, "U0").reshape(-1) for x in U0]
            u = torch.empty(sum(int(p.numel()) for p in parts), dtype=torch.float64, device=parts[0].device)
            off = 0
            for p in parts:
                u[off:off + p.numel()].copy_(p)
                off += p.numel()
    nnz = int(v.numel())
    if tuple(c.shape) != (N, nnz):
        raise ValueError(f"coords must have shape ({N}, {nnz}), got {tuple(c.shape)}")
    u_ptr = None
    if U0 is not None:
        keep.append(u)
        u_ptr = u.data_ptr()
    dims_a = (ctypes.c_int64 * N)(*[int(d) for d in dims])
    ranks_a = (ctypes.c_int * N)(*[int(r) for r in ranks])
    h = ctypes.c_void_p()
    rc = lib.tucker_init(ctypes.byref(h), N, dims_a, nnz, c.data_ptr() if nnz else None,
                         v.data_ptr() if nnz else None, ranks_a, u_ptr, int(seed), flags, _stream(stream))
    _check(rc, "tucker_init")
    return Context(h, dims, ranks, flags)


def ttmc_mode(ctx: Context, mode: int, Y: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if Y is None:
        Y = torch.empty((ctx.dims[mode], ctx.P(mode)), dtype=torch.float32, device="cuda")
    _dev(Y, torch.float32, "Y")
    _check(load().ttmc_mode(ctx.handle, int(mode), Y.data_ptr(), _stream(stream)), "ttmc_mode", ctx)
    return Y


def ttmc_mode_norms(ctx: Context, mode: int, Y: torch.Tensor | None = None, colsq: torch.Tensor | None = None,
                    stream=None):
    """ttmc_mode plus the column sums of squares of Y_(n) (float64 [P_n]) formed as Y is
    written.  Returns (Y, colsq)."""
    if Y is None:
        Y = torch.empty((ctx.dims[mode], ctx.P(mode)), dtype=torch.float32, device="cuda")
    if colsq is None:
        colsq = torch.empty(ctx.P(mode), dtype=torch.float64, device="cuda")
    _dev(Y, torch.float32, "Y")
    _dev(colsq, torch.float64, "colsq")
    _check(load().ttmc_mode_norms(ctx.handle, int(mode), Y.data_ptr(), colsq.data_ptr(), _stream(stream)),
           "ttmc_mode_norms", ctx)
    return Y, colsq


def hooi_iter(ctx: Context, fit_out: torch.Tensor | None = None, stream=None):
    """One HOOI sweep.  Returns the fit as a Python float (synchronises), or writes it
    into the device tensor `fit_out` (float64 [1]) when the context has fit_device."""
    lib = load()
    if ctx.flags & TUCKER_F_FIT_DEVICE:
        if fit_out is None:
            fit_out = torch.empty(1, dtype=torch.float64, device="cuda")
        _check(lib.hooi_iter(ctx.handle, fit_out.data_ptr(), _stream(stream)), "hooi_iter", ctx)
        return fit_out
    f = ctypes.c_double(0.0)
    _check(lib.hooi_iter(ctx.handle, ctypes.addressof(f), _stream(stream)), "hooi_iter", ctx)
    return f.value


def core_tensor(ctx: Context, G: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if G is None:
        G = torch.empty(ctx.ranks, dtype=torch.float64, device="cuda")
    _dev(G, torch.float64, "G")
    _check(load().core_tensor(ctx.handle, G.data_ptr(), _stream(stream)), "core_tensor", ctx)
    return G


def tucker_get_factor(ctx: Context, mode: int, U: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if U is None:
        U = torch.empty((ctx.dims[mode], ctx.ranks[mode]), dtype=torch.float64, device="cuda")
    _dev(U, torch.float64, "U")
    _check(load().tucker_get_factor(ctx.handle, int(mode), U.data_ptr(), _stream(stream)), "tucker_get_factor", ctx)
    return U


def tucker_set_factor(ctx: Context, mode: int, U: torch.Tensor, stream=None) -> None:
    if ctx.flags & TUCKER_F_HOST_INPUT:
        U = torch.as_tensor(np.ascontiguousarray(np.asarray(U.cpu() if isinstance(U, torch.Tensor) else U,
                                                            dtype=np.float64)))
    else:
        _dev(U, torch.float64, "U")
    _check(load().tucker_set_factor(ctx.handle, int(mode), U.data_ptr(), _stream(stream)), "tucker_set_factor", ctx)
    if ctx.flags & TUCKER_F_HOST_INPUT:
        torch.cuda.current_stream().synchronize()


def tucker_loss_grad(ctx: Context, U, G: torch.Tensor, loss=None, dU=None, dG=None, stream=None):
    lib = load()
    N = ctx.N
    U = [_dev(u.contiguous(), torch.float32, "U") for u in U]
    G = _dev(G.contiguous(), torch.float32, "G")
    if loss is None:
        loss = torch.empty(1, dtype=torch.float64, device="cuda")
    if dU is None:
        dU = [torch.empty_like(u) for u in U]
    if dG is None:
        dG = torch.empty_like(G)
    Up = (ctypes.c_void_p * N)(*[u.data_ptr() for u in U])
    dUp = (ctypes.c_void_p * N)(*[d.data_ptr() for d in dU])
    _check(lib.tucker_loss_grad(ctx.handle, Up, G.data_ptr(), loss.data_ptr(), dUp, dG.data_ptr(), _stream(stream)),
           "tucker_loss_grad", ctx)
    return loss, dU, dG


def tucker_nnz(ctx: Context) -> int:
    return int(load().tucker_nnz(ctx.handle))


def tucker_norm2(ctx: Context) -> float:
    return float(load().tucker_norm2(ctx.handle))


def tucker_sync_status(ctx: Context, stream=None) -> None:
    _check(load().tucker_sync_status(ctx.handle, _stream(stream)), "tucker_sync_status", ctx)


def tucker_free(ctx: Context) -> None:
    if ctx.handle:
        load().tucker_free(ctx.handle)
        ctx.handle = None


def tucker_status_str(status: int) -> str:
    return load().tucker_status_str(int(status)).decode()


def tucker_last_error(ctx: Context) -> str:
    return load().tucker_last_error(ctx.handle).decode()


def qrp_leading_work_bytes(m: int, n: int, k: int) -> int:
    return int(load().qrp_leading_work_bytes(int(m), int(n), int(k)))


def qrp_leading(A: torch.Tensor, k: int, work: torch.Tensor | None = None, stream=None):
    """Householder QRP of a device float64 matrix A (m x n, row-major), k reflectors.
    Returns (Q [m, k] float64, piv [k] int64, rdiag [k] float64)."""
    _dev(A, torch.float64, "A")
    m, n = A.shape
    lib = load()
    need = qrp_leading_work_bytes(m, n, k)
    if work is None:
        work = torch.empty(max(need, 256), dtype=torch.uint8, device="cuda")
    Q = torch.empty((m, k), dtype=torch.float64, device="cuda")
    piv = torch.empty(k, dtype=torch.int64, device="cuda")
    rdiag = torch.empty(k, dtype=torch.float64, device="cuda")
    _check(lib.qrp_leading(A.data_ptr(), m, n, n, int(k), Q.data_ptr(), piv.data_ptr(), rdiag.data_ptr(),
                           work.data_ptr(), work.numel(), _stream(stream)), "qrp_leading")
    return Q, piv, rdiag


def qrp_leading_sync_status(work: torch.Tensor, stream=None) -> None:
    """Raise if the last qrp_leading that used `work` gave up a bounded wait or found its
    launch different from its plan (synchronises the stream)."""
    _check(load().qrp_leading_sync_status(work.data_ptr(), _stream(stream)), "qrp_leading_sync_status")


def qrp_leading_noalloc_sync_status(stream=None) -> None:
    _check(load().qrp_leading_noalloc_sync_status(_stream(stream)), "qrp_leading_noalloc_sync_status")


def tucker_set_profiling(ctx: Context, enable: bool = True) -> None:
    _check(load().tucker_set_profiling(ctx.handle, int(bool(enable))), "tucker_set_profiling", ctx)


def tucker_phase_times(ctx: Context):
    """Per-phase milliseconds of the latest profiled sweep: [ttmc_1, qrp_1, ..., ttmc_N, qrp_N, core]."""
    n = 2 * ctx.N + 1
    buf = (ctypes.c_float * n)()
    got = load().tucker_phase_times(ctx.handle, buf, n)
    if got != n:
        raise TuckerError(6, "tucker_phase_times", "profiling off or no complete sweep")
    return [float(x) for x in buf]


MODE_INFO_KEYS = ("slices", "chunk", "units", "long_slices", "fibers_on", "fibers", "fchunk", "fiber_units",
                  "fiber_long_slices", "fiber_cap", "fiber_mid_mode")


def tucker_mode_info(ctx: Context, mode: int) -> dict:
    """Layout of one mode's sorted copy: slices, work units, fiber level (instrumentation)."""
    buf = (ctypes.c_int64 * len(MODE_INFO_KEYS))()
    got = load().tucker_mode_info(ctx.handle, int(mode), buf, len(MODE_INFO_KEYS))
    if got != len(MODE_INFO_KEYS):
        raise TuckerError(1, "tucker_mode_info")
    return {k: int(v) for k, v in zip(MODE_INFO_KEYS, buf)}


def tucker_hooi_graph(ctx: Context, sweeps: int, fit: torch.Tensor, stream=None) -> None:
    """`sweeps` HOOI sweeps replayed from a CUDA graph of one sweep; the fit of each sweep
    goes to the device float64 tensor `fit` (the same tensor on every call).  `stream` must
    not be the legacy default stream (a torch.cuda.Stream, say)."""
    _dev(fit, torch.float64, "fit")
    if stream is None:
        stream = torch.cuda.current_stream()
    if _stream(stream) == 0:
        raise ValueError("tucker_hooi_graph: a stream other than the legacy default stream is needed")
    _check(load().tucker_hooi_graph(ctx.handle, int(sweeps), fit.data_ptr(), _stream(stream)), "tucker_hooi_graph",
           ctx)


def tucker_fp32_fma_tflops(iters: int = 20000, stream=None) -> float:
    """Measured FP32 FMA throughput of the current GPU (TFLOP/s)."""
    v = float(load().tucker_fp32_fma_tflops(int(iters), _stream(stream)))
    if v <= 0:
        raise TuckerError(4, "tucker_fp32_fma_tflops")
    return v


def tucker_kernel_launches() -> int:
    return int(load().tucker_kernel_launches())


def tucker_check_site() -> int:
    """Checked build: the first index check of the cluster QRP that failed (0: none); -1 in
    the normal build."""
    return int(load().tucker_check_site())


def qrp_leading_noalloc_max_bytes() -> int:
    return int(load().qrp_leading_noalloc_max_bytes())


def qrp_leading_noalloc(A: torch.Tensor, k: int, stream=None):
    """qrp_leading with the library's fixed device scratch (no scratch argument, no
    device allocation inside the call).  Returns (Q, piv, rdiag) like qrp_leading."""
    _dev(A, torch.float64, "A")
    m, n = A.shape
    Q = torch.empty((m, k), dtype=torch.float64, device="cuda")
    piv = torch.empty(k, dtype=torch.int64, device="cuda")
    rdiag = torch.empty(k, dtype=torch.float64, device="cuda")
    _check(load().qrp_leading_noalloc(A.data_ptr(), m, n, n, int(k), Q.data_ptr(), piv.data_ptr(), rdiag.data_ptr(),
                                      _stream(stream)), "qrp_leading_noalloc")
    return Q, piv, rdiag


def tucker_selftest_wait(ctx: Context, max_polls: int, stream=None) -> None:
    _check(load().tucker_selftest_wait(ctx.handle, int(max_polls), _stream(stream)), "tucker_selftest_wait", ctx)


def tucker_selftest_sort_wait(max_polls: int, stream=None) -> str:
    """Runs the sort's bounded look-back self-test; returns the status name
    ("TUCKER_ETIMEOUT" when the wait gave up as designed)."""
    rc = load().tucker_selftest_sort_wait(int(max_polls), _stream(stream))
    if rc not in (0, 5):
        _check(rc, "tucker_selftest_sort_wait")
    return STATUS[rc]
