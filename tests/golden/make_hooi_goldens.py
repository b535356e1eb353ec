"""Write the stored HOOI results of the full-size workload recipes (tests/golden/hooi_<name>.json).

    python tests/golden/make_hooi_goldens.py order4-5M skew-20M [zipf-10k^3 ...]

Every number written here comes from the FP64 oracle (``oracle/``) on the seeded inputs
of ``paper_2010_10638_gb300.synth``; nothing is taken from the CUDA library.  One record
per workload:

  fits         fit after every sweep (Algorithm 2, fixed sweep count of the recipe)
  pivots       per sweep and mode, the columns QRP chose (Section III-D)
  rdiag        per sweep and mode, the diagonal of R (|r_11| >= ... >= |r_kk|); the ratio
               |r_11 / r_kk| bounds how much a perturbation of the factored matrix can turn
               the last column of Q
  min_gap      per sweep and mode, the smallest relative gap between the largest and the
               second-largest trailing column norm over the R_n pivot decisions (exact
               norms of the matrix QRP factored); a pivot decision closer than the FP32
               rounding of Y_(n) can go either way on an FP32 path
  G_canon      the core of the last sweep with every factor column's sign fixed by the
               sign of its largest-magnitude entry (C-order, flattened)
  sketch       per mode, the sign-fixed U_n^T W_n (R_n x 4) with W_n seeded N(0, 1) rows
               (numpy default_rng(7 + n)), a fingerprint of the factor itself

The sign convention and the sketch (tests/hooi_canon.py) are applied the same way to the
GPU's factors in tests/test_gpu_hooi_full.py.
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2010_10638_gb300 import synth  # noqa: E402
from tests.hooi_canon import canonical, sketch  # noqa: E402


def min_pivot_gap(A, res, k):
    """Smallest relative gap between the top two trailing column norms over k pivot steps,
    from the oracle's own pivots and reflectors (trailing norms = norms of the components
    orthogonal to the pivot columns chosen so far)."""
    n = A.shape[1]
    rest = [c for c in range(n) if c not in set(res.piv.tolist())]
    W = A[:, np.concatenate([res.piv, rest]).astype(int)]
    gaps = []
    for j in range(k):
        Qj = res.Q[:, :j]
        R = W[:, j:] - Qj @ (Qj.T @ W[:, j:])
        nrm = np.sort(np.linalg.norm(R, axis=0))[::-1]
        if len(nrm) > 1 and nrm[0] > 0:
            gaps.append(float((nrm[0] - nrm[1]) / nrm[0]))
    return min(gaps) if gaps else 1.0


def oracle_sweeps(inst, iters=None, log=None, threads=1):
    """Algorithm 2 by the oracle's routines, recording per sweep and mode the pivots, the R
    diagonal and the smallest pivot gap; returns (record, U, G) with U and G of the last sweep."""
    w = inst.workload
    dims, ranks, N = w.dims, w.ranks, len(w.dims)
    iters = w.iters if iters is None else iters
    t0 = time.time()
    cc, cv = oracle.coalesce(inst.coords, inst.vals.astype(np.float64))
    nx2 = oracle.norm2(cv)
    U = [None] + [np.asarray(inst.U0[m], dtype=np.float64) for m in range(1, N)]
    fits, pivots, rdiags, gaps = [], [], [], []
    G = None
    for it in range(iters):
        pv, rd, gp = [], [], []
        for n in range(N):
            Y = oracle.ttmc(dims, ranks, cc, cv, n, U, threads)
            A = Y if Y.shape[1] <= Y.shape[0] else oracle.gram(Y, threads)
            res = oracle.qrp(A, ranks[n], threads)
            U[n] = res.Q
            pv.append([int(x) for x in res.piv])
            rd.append([float(x) for x in res.rdiag])
            gp.append(min_pivot_gap(A, res, ranks[n]))
        G = oracle.core(Y, U[N - 1], ranks, threads)
        fits.append(oracle.fit_from_core(nx2, G))
        pivots.append(pv)
        rdiags.append(rd)
        gaps.append(gp)
        if log:
            log(f"{w.name}: sweep {it + 1}/{iters} fit {fits[-1]:.12f} min gap {min(gp):.2e} "
                f"({time.time() - t0:.0f} s)")
    rec = {"workload": w.name, "dims": list(dims), "nnz_listed": w.nnz, "nnz_coalesced": int(cc.shape[1]),
           "ranks": list(ranks), "sweeps": iters, "seed": w.seed, "normX2": nx2, "fits": fits,
           "pivots": pivots, "rdiag": rdiags, "min_gap": gaps}
    return rec, U, G


def run(name):
    inst = synth.make(name)
    N = len(inst.workload.dims)
    t0 = time.time()
    rec, U, G = oracle_sweeps(inst, log=lambda m: print(m, flush=True))
    Uc, Gc = canonical(U, G)
    rec.update({"G_canon": [float(x) for x in Gc.reshape(-1)],
                "sketch": [[[float(x) for x in row] for row in sketch(Uc[n], n)] for n in range(N)],
                "command": f"python tests/golden/make_hooi_goldens.py {name}",
                "source": "FP64 oracle (oracle/tucker_oracle.c via oracle/oracle.py), Algorithm 2 with QRP"})
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"hooi_{name}.json")
    with open(out, "w") as f:
        json.dump(rec, f, indent=0)
    print(f"wrote {out} ({time.time() - t0:.0f} s)")


if __name__ == "__main__":
    for nm in sys.argv[1:]:
        run(nm)
