"""A HOOI sweep captured once as a CUDA graph and replayed (tucker_hooi_graph) gives the
same fits, factors and core as the same number of hooi_iter calls, bit for bit (the graph
runs the same kernels in the same order on the same data)."""
import numpy as np
import pytest

from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, torch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,nnz,bf16", [("skew-20M", 300_000, False), ("order4-5M", 200_000, False),
                                           ("zipf-10k^3", 200_000, True)])
def test_graph_sweeps_equal_eager_sweeps(name, nnz, bf16):
    T = lib()
    inst = synth.make(name, nnz=nnz)
    w = inst.workload
    args = (w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(), torch.as_tensor(inst.vals).cuda(), w.ranks,
            [torch.as_tensor(u).cuda() for u in inst.U0])
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        a = T.tucker_init(*args, bf16=bf16, stream=stream)
        b = T.tucker_init(*args, bf16=bf16, stream=stream)
        fits_a = [T.hooi_iter(a, stream=stream) for _ in range(4)]
        fit = torch.zeros(1, dtype=torch.float64, device="cuda")
        fits_b = []
        for _ in range(2):  # the first call runs one sweep eagerly and captures the next
            T.tucker_hooi_graph(b, 1, fit, stream=stream)
            stream.synchronize()
            fits_b.append(float(fit.item()))
        before = T.tucker_kernel_launches()
        T.tucker_hooi_graph(b, 2, fit, stream=stream)  # two replays in one call
        stream.synchronize()
        per_sweep = (T.tucker_kernel_launches() - before) / 2
        assert per_sweep >= 3 * len(w.dims)  # every replay counts its kernels (TTMc, QRP, refresh per mode)
        fits_b.append(float("nan"))
        fits_b.append(float(fit.item()))
        assert fits_a[:2] == fits_b[:2] and fits_a[3] == fits_b[3]
        for n in range(len(w.dims)):
            assert torch.equal(T.tucker_get_factor(a, n), T.tucker_get_factor(b, n))
        assert torch.equal(T.core_tensor(a), T.core_tensor(b))
        T.tucker_sync_status(b, stream=stream)
        T.tucker_free(a)
        T.tucker_free(b)
