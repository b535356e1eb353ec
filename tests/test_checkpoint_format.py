"""Checkpoint files on the CPU: a file that is not a HOOI checkpoint, or one saved for
other dimensions or ranks, is refused before anything touches the device."""
import types

import pytest

torch = pytest.importorskip("torch")


def fake_ctx(dims, ranks):
    return types.SimpleNamespace(dims=tuple(dims), ranks=tuple(ranks), N=len(dims), handle=None, flags=0)


def test_foreign_file_is_refused(tmp_path):
    from paper_2010_10638_gb300 import checkpoint
    p = tmp_path / "other.pt"
    torch.save({"format": "something else"}, p)
    with pytest.raises(ValueError, match="not a HOOI checkpoint"):
        checkpoint.load(fake_ctx((10, 10, 10), (2, 2, 2)), p)
    torch.save([1, 2, 3], p)
    with pytest.raises(ValueError, match="not a HOOI checkpoint"):
        checkpoint.load(fake_ctx((10, 10, 10), (2, 2, 2)), p)


def test_other_dims_or_ranks_are_refused(tmp_path):
    from paper_2010_10638_gb300 import checkpoint
    p = tmp_path / "run.pt"
    torch.save({"format": checkpoint.FORMAT, "dims": [10, 10, 10], "ranks": [2, 2, 2], "nnz": 5, "norm2": 1.0,
                "flags": 0, "sweeps": 1, "fits": [0.5], "factors": [], "core": None}, p)
    with pytest.raises(ValueError, match="ranks"):
        checkpoint.load(fake_ctx((10, 10, 10), (3, 2, 2)), p)
    with pytest.raises(ValueError, match="dims"):
        checkpoint.load(fake_ctx((10, 10, 11), (2, 2, 2)), p)
