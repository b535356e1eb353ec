"""Helpers shared by the GPU parity tests (inputs only; no arithmetic of the method)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def lib():
    need_gpu()
    from paper_2010_10638_gb300 import build, tucker
    build.build()
    tucker.load()
    return tucker


def f32_round(U):
    """Factors as the kernels see them: FP32 copies of the FP64 masters, back in FP64."""
    return [np.asarray(u, dtype=np.float64).astype(np.float32).astype(np.float64) for u in U]


def rel_fro(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))
