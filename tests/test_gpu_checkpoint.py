"""Checkpoint / resume of a HOOI run: sweeps after a resume reproduce an uninterrupted run
bit for bit (the kernels are deterministic), and a checkpoint is refused by a context
built from another tensor or with other ranks."""
import numpy as np
import pytest

from paper_2010_10638_gb300 import synth
from tests.gpu_util import lib, torch

pytestmark = pytest.mark.gpu


def make_ctx(T, inst, ranks=None):
    w = inst.workload
    U0 = None if ranks else [torch.as_tensor(u).cuda() for u in inst.U0]  # other ranks: seeded factors
    return T.tucker_init(w.dims, torch.as_tensor(inst.coords.astype(np.int32)).cuda(),
                         torch.as_tensor(inst.vals).cuda(), ranks or w.ranks, U0)


@pytest.mark.parametrize("name,nnz", [("zipf-10k^3", 200_000), ("skew-20M", 300_000)])
def test_resume_reproduces_uninterrupted_run(tmp_path, name, nnz):
    T = lib()
    from paper_2010_10638_gb300 import checkpoint
    inst = synth.make(name, nnz=nnz)
    a = make_ctx(T, inst)
    fits_a = [T.hooi_iter(a) for _ in range(4)]
    Ua = [T.tucker_get_factor(a, n).cpu().numpy() for n in range(3)]
    Ga = T.core_tensor(a).cpu().numpy()

    b = make_ctx(T, inst)
    fits_b = [T.hooi_iter(b) for _ in range(2)]
    path = tmp_path / "run.pt"
    checkpoint.save(b, path, sweeps=2, fits=fits_b)
    T.tucker_free(b)

    c = make_ctx(T, inst)
    state = checkpoint.load(c, path)
    assert state["sweeps"] == 2 and state["fits"] == fits_b
    fits_c = state["fits"] + [T.hooi_iter(c) for _ in range(2)]
    assert fits_c == fits_a
    for n in range(3):
        np.testing.assert_array_equal(T.tucker_get_factor(c, n).cpu().numpy(), Ua[n])
    np.testing.assert_array_equal(T.core_tensor(c).cpu().numpy(), Ga)


def test_checkpoint_refused_for_another_tensor_or_ranks(tmp_path):
    T = lib()
    from paper_2010_10638_gb300 import checkpoint
    inst = synth.make("tiny-100^3")
    a = make_ctx(T, inst)
    T.hooi_iter(a)
    path = tmp_path / "tiny.pt"
    checkpoint.save(a, path, sweeps=1)
    other = synth.make("tiny-100^3", seed=77)  # same shape, other entries
    with pytest.raises(ValueError, match="another tensor"):
        checkpoint.load(make_ctx(T, other), path)
    with pytest.raises(ValueError, match="ranks"):
        checkpoint.load(make_ctx(T, inst, ranks=(4, 4, 4)), path)
    torch.save({"format": "something else"}, tmp_path / "bad.pt")
    with pytest.raises(ValueError, match="not a HOOI checkpoint"):
        checkpoint.load(a, tmp_path / "bad.pt")
