"""Small, fixed workloads for profiling one kernel family under a profiler (ncu).

    python -m paper_2010_10638_gb300.profile_driver ttmc MODE [--nnz N] [--bf16] [--reps R]
    python -m paper_2010_10638_gb300.profile_driver qrp [--nnz N]

`ttmc` builds the skew-20M recipe at N nonzeros (default 12M: the nonzero stream is
larger than L2, and the device footprint stays near 1 GB) and runs ttmc_mode(MODE) R
times; `qrp` runs one HOOI sweep on the same recipe at 2M nonzeros (the QRP size depends
only on the unfolding, 50,000 x 256 for modes 1-2).  Profile with, e.g.,

    ncu --set full --clock-control none -k regex:ttmc_pipe -s 1 -c 1 -o out \\
        python -m paper_2010_10638_gb300.profile_driver ttmc 1
"""
from __future__ import annotations

import argparse

import numpy as np
import torch

from . import synth
from . import tucker as T


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["ttmc", "qrp"])
    ap.add_argument("mode", nargs="?", type=int, default=0)
    ap.add_argument("--nnz", type=int, default=None)
    ap.add_argument("--bf16", action="store_true")
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    T.load()
    nnz = a.nnz or (12_000_000 if a.what == "ttmc" else 2_000_000)
    w = synth.make("skew-20M", nnz=nnz)
    ctx = T.tucker_init(w.workload.dims, torch.as_tensor(w.coords.astype(np.int32)).cuda(),
                        torch.as_tensor(w.vals).cuda(), w.workload.ranks, [torch.as_tensor(u).cuda() for u in w.U0],
                        bf16=a.bf16)
    if a.what == "ttmc":
        Y = torch.empty((w.workload.dims[a.mode], ctx.P(a.mode)), device="cuda")
        for _ in range(a.reps):
            T.ttmc_mode(ctx, a.mode, Y)
    else:
        T.hooi_iter(ctx)
    torch.cuda.synchronize()
    print("ok", T.tucker_nnz(ctx))


if __name__ == "__main__":
    main()
