"""Seeded synthetic sparse tensors shaped like the workloads of arXiv 2010.10638.

This module only draws inputs.  It holds none of the method's arithmetic (no TTMc,
no QRP, no core tensor, no loss); the CUDA path and the FP64 oracle both take their
inputs from here and from nowhere else.

Workloads (the paper's own datasets are not available; these stand in for them):

  tiny-100^3     order 3, 100x100x100, 10,000 distinct uniform coordinates,
                 values U(0,1), ranks (8,8,8), 5 sweeps
  zipf-10k^3     order 3, 10,000^3, 1M coordinates Zipf(1.1) in every mode,
                 values U(0,1), ranks (16,16,16), 10 sweeps
  order4-5M      order 4, 5000x5000x2000x500, 5M uniform coordinates,
                 values N(0,1), ranks (8,8,8,8), 10 sweeps
  skew-20M       order 3, 50,000x50,000x1,000, 20M coordinates, Zipf(1.2) in
                 mode 1 and uniform in modes 2-3, values lognormal(0,1),
                 ranks (16,16,16), 10 sweeps
  completion-10M order 3, 20,000^3, 10M uniform coordinates, values from a seeded
                 rank-(10,10,10) Tucker model plus N(0, 0.01^2) noise

Zipf(s) on [0, I): P(i) proportional to (i+1)^-s, followed by a seeded random
relabelling of the indices so that the heavy slices are not adjacent.  Coordinates
are drawn independently per mode (duplicates can occur and are summed at init),
except tiny-100^3 whose coordinates are distinct.  Every workload uses
numpy.random.default_rng(seed) with seed = 1000 + its index (1..5).

Initial factors: U_m ~ N(0,1) of shape I_m x R_m, orthonormalised by LAPACK's
unpivoted Householder QR (numpy.linalg.qr); identical copies go to both sides.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Workload:
    name: str
    dims: tuple
    nnz: int
    ranks: tuple
    iters: int
    seed: int
    coord_dist: tuple        # per mode: ("uniform",) or ("zipf", s); ("distinct",) for all modes
    value_dist: str          # "uniform" | "normal" | "lognormal" | "tucker"
    noise_sigma: float = 0.0
    notes: str = ""
    extra: dict = field(default_factory=dict)


WORKLOADS = {
    "tiny-100^3": Workload("tiny-100^3", (100, 100, 100), 10_000, (8, 8, 8), 5, 1001,
                           ("distinct",), "uniform"),
    "zipf-10k^3": Workload("zipf-10k^3", (10_000, 10_000, 10_000), 1_000_000, (16, 16, 16), 10, 1002,
                           (("zipf", 1.1), ("zipf", 1.1), ("zipf", 1.1)), "uniform"),
    "order4-5M": Workload("order4-5M", (5000, 5000, 2000, 500), 5_000_000, (8, 8, 8, 8), 10, 1003,
                          (("uniform",),) * 4, "normal"),
    "skew-20M": Workload("skew-20M", (50_000, 50_000, 1_000), 20_000_000, (16, 16, 16), 10, 1004,
                         (("zipf", 1.2), ("uniform",), ("uniform",)), "lognormal"),
    "completion-10M": Workload("completion-10M", (20_000, 20_000, 20_000), 10_000_000, (10, 10, 10), 1, 1005,
                               (("uniform",),) * 3, "tucker", noise_sigma=0.01),
}


# Section IV-C, Fig. 7: 200 x 200 x 200 random tensors of varying sparsity, ranks 16 (the
# figure's sparsity values are not printed; this grid spans 1e-4 .. 0.3).
FIG7_DENSITIES = (1e-4, 1e-3, 1e-2, 3e-2, 1e-1, 3e-1)


def fig7_workload(i: int) -> Workload:
    d = FIG7_DENSITIES[i]
    return Workload(f"fig7-200^3-d{d:g}", (200, 200, 200), int(round(d * 200 ** 3)), (16, 16, 16), 5, 1100 + i,
                    ("distinct",), "uniform")


# Table III: the dense tensor-times-matrix of the core step, a 32 x 32 x I3 tensor times a
# 32 x I3 factor, I3 = 32 .. 256 (all entries listed as nonzeros, ranks 32).
TABLE3_I3 = (32, 64, 128, 256)


def table3_workload(i: int) -> Workload:
    i3 = TABLE3_I3[i]
    return Workload(f"table3-32x32x{i3}", (32, 32, i3), 32 * 32 * i3, (32, 32, 32), 1, 1200 + i, ("distinct",),
                    "normal")


def zipf_indices(rng, n: int, size: int, s: float) -> np.ndarray:
    """Draw `size` indices on [0, n) with P(i) ~ (i+1)^-s, then relabel by a seeded permutation."""
    w = (np.arange(1, n + 1, dtype=np.float64)) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    u = rng.random(size)
    rank = np.minimum(np.searchsorted(cdf, u, side="right"), n - 1)
    relabel = rng.permutation(n)
    return relabel[rank].astype(np.uint32)


def orthonormal_factor(rng, rows: int, cols: int) -> np.ndarray:
    g = rng.standard_normal((rows, cols))
    q, _ = np.linalg.qr(g)
    return np.ascontiguousarray(q, dtype=np.float64)


def draw_coords(rng, w: Workload) -> np.ndarray:
    N = len(w.dims)
    if w.coord_dist == ("distinct",):
        total = int(np.prod(w.dims, dtype=np.int64))
        flat = rng.choice(total, size=w.nnz, replace=False)
        return np.stack(np.unravel_index(flat, w.dims)).astype(np.uint32)
    coords = np.empty((N, w.nnz), dtype=np.uint32)
    for m in range(N):
        d = w.coord_dist[m]
        if d[0] == "uniform":
            coords[m] = rng.integers(0, w.dims[m], size=w.nnz, dtype=np.uint32)
        elif d[0] == "zipf":
            coords[m] = zipf_indices(rng, w.dims[m], w.nnz, d[1])
        else:
            raise ValueError(d)
    return coords


@dataclass
class Instance:
    workload: Workload
    coords: np.ndarray       # uint32 [N, nnz], 0-based
    vals: np.ndarray         # float32 [nnz]
    U0: list                 # float64 I_m x R_m, orthonormal columns
    model: dict | None = None  # generating Tucker model for "tucker" values


def make(name_or_workload, nnz: int | None = None, seed: int | None = None) -> Instance:
    """Draw one workload.  `nnz` and `seed` override the recipe (smaller parity cases)."""
    w = WORKLOADS[name_or_workload] if isinstance(name_or_workload, str) else name_or_workload
    if nnz is not None or seed is not None:
        w = Workload(**{**w.__dict__, "nnz": nnz if nnz is not None else w.nnz,
                        "seed": seed if seed is not None else w.seed})
    rng = np.random.default_rng(w.seed)
    coords = draw_coords(rng, w)
    model = None
    if w.value_dist == "uniform":
        vals = rng.random(w.nnz, dtype=np.float32)
    elif w.value_dist == "normal":
        vals = rng.standard_normal(w.nnz, dtype=np.float32)
    elif w.value_dist == "lognormal":
        vals = rng.lognormal(0.0, 1.0, size=w.nnz).astype(np.float32)
    elif w.value_dist == "tucker":
        vals, model = tucker_model_values(rng, w.dims, w.ranks, coords, w.noise_sigma)
    else:
        raise ValueError(w.value_dist)
    U0 = [orthonormal_factor(rng, w.dims[m], w.ranks[m]) for m in range(len(w.dims))]
    return Instance(w, coords, vals, U0, model)


def tucker_model_values(rng, dims, ranks, coords, sigma, chunk=1 << 20):
    """Values of a seeded Tucker model at the given coordinates, plus N(0, sigma^2) noise.
    Model: U_m ~ N(0,1) (I_m x R_m), G ~ N(0, 1/prod R) so that Var(x) is about 1."""
    N = len(dims)
    Um = [rng.standard_normal((dims[m], ranks[m])) for m in range(N)]
    G = rng.standard_normal(tuple(ranks)) / np.sqrt(float(np.prod(ranks)))
    nnz = coords.shape[1]
    vals = np.empty(nnz, dtype=np.float64)
    for s in range(0, nnz, chunk):
        e = min(nnz, s + chunk)
        t = G.reshape(ranks[0], -1)
        acc = Um[0][coords[0, s:e]] @ t  # [c, prod R_2..R_N]
        for m in range(1, N):
            acc = acc.reshape(e - s, ranks[m], -1)
            acc = np.einsum("zr,zrq->zq", Um[m][coords[m, s:e]], acc)
        vals[s:e] = acc.reshape(-1)
    vals += sigma * rng.standard_normal(nnz)
    return vals.astype(np.float32), {"U": Um, "G": G}


def random_factors(rng, dims, ranks, orthonormal=True, dtype=np.float64):
    """Factors for kernel-level parity cases (the same arrays go to both sides)."""
    out = []
    for d, r in zip(dims, ranks):
        out.append(orthonormal_factor(rng, d, r) if orthonormal else rng.standard_normal((d, r)))
    return [np.ascontiguousarray(u, dtype=dtype) for u in out]


def pmm_tensor(M=5, K=5, N=5):
    """Binary tensor of the classical matrix product C = A B (Section IV-C, PMM):
    x(i1, i2, i3) = 1 when entry i1 of A (row-major M x K) times entry i2 of B
    (row-major K x N) is accumulated into entry i3 of C (column-major M x N)."""
    cs = []
    for m in range(M):
        for k in range(K):
            for n in range(N):
                cs.append((m * K + k, k * N + n, n * M + m))
    coords = np.array(cs, dtype=np.uint32).T.copy()
    vals = np.ones(coords.shape[1], dtype=np.float32)
    return (M * K, K * N, M * N), coords, vals


def low_rank_dense(rng, dims, ranks):
    """A dense tensor of exact multilinear rank `ranks` (random core, orthonormal
    factors), returned with all of its entries as COO (for exact-recovery cases)."""
    N = len(dims)
    G = rng.standard_normal(tuple(ranks))
    Us = [orthonormal_factor(rng, dims[m], ranks[m]) for m in range(N)]
    X = G
    for m in range(N):
        X = np.tensordot(Us[m], X, axes=([1], [m]))
        X = np.moveaxis(X, 0, m)
    idx = np.indices(dims).reshape(N, -1).astype(np.uint32)
    return X, idx, X.reshape(-1).astype(np.float64)
