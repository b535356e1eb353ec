"""Checkpoint and resume of a HOOI run (Algorithm 2).

The state of a run between sweeps is its factor matrices U_1 .. U_N (FP64; every sweep
reads only these), the number of sweeps done and the fit history.  `save` writes them
with torch.save together with the tensor's dimensions, ranks, nonzero count and squared
norm; `load` checks those against the context it restores into (a context built from
the same tensor) and sets the factors.  The kernels are deterministic (no atomics, fixed
summation orders), so sweeps after a resume reproduce an uninterrupted run bit for bit.

    ckpt = checkpoint.save(ctx, "run.pt", sweeps=5, fits=fits)
    ...
    ctx2 = tucker.tucker_init(dims, coords, vals, ranks)        # same tensor
    state = checkpoint.load(ctx2, "run.pt")                     # state["sweeps"], state["fits"]
"""
from __future__ import annotations

import torch

from . import tucker as T

FORMAT = "tucker-hooi-checkpoint/1"


def save(ctx: T.Context, path, sweeps: int, fits=(), stream=None) -> dict:
    """Write the factors of `ctx` and the run's progress to `path`; returns the saved dict."""
    factors = [T.tucker_get_factor(ctx, n, stream=stream).cpu() for n in range(ctx.N)]
    try:
        G = T.core_tensor(ctx, stream=stream).cpu()
    except T.TuckerError:  # no sweep since the factors were set: no core to keep
        G = None
    state = {"format": FORMAT, "dims": list(ctx.dims), "ranks": list(ctx.ranks), "nnz": T.tucker_nnz(ctx),
             "norm2": T.tucker_norm2(ctx), "flags": int(ctx.flags), "sweeps": int(sweeps),
             "fits": [float(f) for f in fits], "factors": factors, "core": G}
    torch.save(state, path)
    return state


def load(ctx: T.Context, path, stream=None) -> dict:
    """Restore the factors saved at `path` into `ctx` (built from the same tensor and
    ranks); returns the saved state (sweeps done, fit history, core)."""
    state = torch.load(path, weights_only=False)
    if not isinstance(state, dict) or state.get("format") != FORMAT:
        raise ValueError(f"{path}: not a HOOI checkpoint")
    if list(ctx.dims) != state["dims"] or list(ctx.ranks) != state["ranks"]:
        raise ValueError(f"{path}: saved for dims {state['dims']} ranks {state['ranks']}, "
                         f"context has dims {list(ctx.dims)} ranks {list(ctx.ranks)}")
    if T.tucker_nnz(ctx) != state["nnz"] or T.tucker_norm2(ctx) != state["norm2"]:
        raise ValueError(f"{path}: saved for another tensor (nonzero count or norm differs)")
    dev = torch.device("cuda", torch.cuda.current_device())
    for n, U in enumerate(state["factors"]):
        T.tucker_set_factor(ctx, n, U.to(device=dev, dtype=torch.float64).contiguous(), stream=stream)
    return state
