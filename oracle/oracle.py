"""FP64 CPU oracle for sparse Tucker / HOOI with QR column pivoting (arXiv 2010.10638).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's CPU-baseline leg
may import this module; the product library never does, and the two share no code.

The arithmetic lives in ``tucker_oracle.c`` (plain loops, double precision); this
module compiles and loads it with ``ctypes``, adapts numpy arrays, and drives the
HOOI sweep of Algorithm 2 step by step:

    for each sweep:
        for n = 1..N:   Y_(n) = TTMc(X, {U_m}_{m != n})        (Alg. 2, Kronecker accumulate)
                        U_n   = QRP(Y_(n), R_n)[:, :R_n]          (Alg. 2, Section III-D)
        G = U_N^T Y_(N)                                           (Alg. 2, eq. core_unfolded)
        fit = 1 - sqrt(max(0, ||X||^2 - ||G||^2)) / ||X||

Functions and the passage each follows:
  coalesce      - COO with duplicate coordinates summed (Section III-A, Table I)
  ttmc          - Alg. 2 inner loop / Section III-C eq. for Y_(1), Alg. 4 layout
  qrp           - Section III-D (A P = Q R, Householder reflectors, column norms each step)
  gram          - Section III-D, fat case: QRP on Y Y^T
  core          - Section III-B, eqs. ttm_ele and core_unfolded
  hooi          - Algorithm 2; ``svd=True`` swaps QRP for the SVD of Algorithm 1 (check only)
  loss_grad     - observed-entry loss 1/2 sum (x - [[G; U]])^2 and its gradients
  kron_count    - Kronecker rows formed so far (one per nonzero per mode, Section IV-C)

``threads > 1`` (ttmc, qrp, gram, core, hooi) runs ``tucker_oracle_par.c``: the same loops
split over POSIX threads by output column, equal to the serial results bit for bit (a CPU
test checks this); it exists to time the oracle on all of a machine's cores.

Parity status: every function above is pinned by tests under ``tests/`` against
dense brute force, closed forms, LAPACK (scipy) or printed values of the paper.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tucker_oracle.c")
_SRC_PAR = os.path.join(_HERE, "tucker_oracle_par.c")  # the same routines split over threads by column
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libtucker_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc -O2, no fast-math) into oracle/_build/."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC_PAR))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-o", tmp, _SRC, _SRC_PAR,
                               "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        c_i64, c_int, c_dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_coalesce.restype = c_i64
        lib.orc_coalesce.argtypes = [c_int, c_i64, P(ctypes.c_uint32), P(c_dbl), P(ctypes.c_uint32), P(c_dbl)]
        lib.orc_ttmc.restype = None
        lib.orc_ttmc.argtypes = [c_int, P(c_i64), P(c_int), c_i64, P(ctypes.c_uint32), P(c_dbl), c_int,
                                 P(P(c_dbl)), P(c_dbl)]
        lib.orc_qrp.restype = c_int
        lib.orc_qrp.argtypes = [P(c_dbl), c_i64, c_i64, c_i64, c_int, P(c_dbl), P(c_i64), P(c_dbl)]
        lib.orc_gram.restype = None
        lib.orc_gram.argtypes = [P(c_dbl), c_i64, c_i64, P(c_dbl)]
        lib.orc_core.restype = None
        lib.orc_core.argtypes = [c_i64, c_i64, c_int, P(c_dbl), P(c_dbl), P(c_dbl)]
        lib.orc_loss_grad.restype = None
        lib.orc_loss_grad.argtypes = [c_int, P(c_i64), P(c_int), c_i64, P(ctypes.c_uint32), P(c_dbl),
                                      P(P(c_dbl)), P(c_dbl), P(c_dbl), P(P(c_dbl)), P(c_dbl)]
        lib.orc_ttmc_par.restype = None
        lib.orc_ttmc_par.argtypes = [c_int, P(c_i64), P(c_int), c_i64, P(ctypes.c_uint32), P(c_dbl), c_int,
                                     P(P(c_dbl)), P(c_dbl), c_int]
        lib.orc_qrp_par.restype = c_int
        lib.orc_qrp_par.argtypes = [P(c_dbl), c_i64, c_i64, c_i64, c_int, P(c_dbl), P(c_i64), P(c_dbl), c_int]
        lib.orc_gram_par.restype = None
        lib.orc_gram_par.argtypes = [P(c_dbl), c_i64, c_i64, P(c_dbl), c_int]
        lib.orc_core_par.restype = None
        lib.orc_core_par.argtypes = [c_i64, c_i64, c_int, P(c_dbl), P(c_dbl), P(c_dbl), c_int]
        lib.orc_kron_count.restype = c_i64
        lib.orc_kron_count.argtypes = []
        lib.orc_kron_reset.restype = None
        lib.orc_kron_reset.argtypes = []
        _lib = lib
    return _lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def _ptr_array(mats):
    arr = (ctypes.POINTER(ctypes.c_double) * len(mats))()
    for i, m in enumerate(mats):
        arr[i] = _ptr(m, ctypes.c_double)
    return arr


# --------------------------------------------------------------------------- COO
def coalesce(coords, vals):
    """Sum duplicate coordinates (FP64).  coords: [N, nnz] integer, vals: [nnz].
    Returns (coords u32 [N, nnz'], vals f64 [nnz']) sorted by full coordinate."""
    lib = _load()
    coords = _u32(coords)
    vals = _f64(vals)
    N, nnz = coords.shape
    oc = np.zeros((N, max(nnz, 1)), dtype=np.uint32).reshape(-1)
    ov = np.zeros(max(nnz, 1), dtype=np.float64)
    out = lib.orc_coalesce(N, nnz, _ptr(coords, ctypes.c_uint32), _ptr(vals, ctypes.c_double),
                           _ptr(oc, ctypes.c_uint32), _ptr(ov, ctypes.c_double))
    return oc[: N * out].reshape(N, out).copy(), ov[:out].copy()


def norm2(vals) -> float:
    """||X||_F^2 of a coalesced COO tensor (Definition 2)."""
    v = _f64(vals)
    return float(np.sum(v * v))


# --------------------------------------------------------------------------- TTMc
def ttmc(dims, ranks, coords, vals, mode, U, threads=1):
    """Y_(mode) = X_(mode) (kron_{m != mode} U_m), Alg. 2 inner loop, FP64.
    Y is [I_mode, P] with the remaining modes ascending, last fastest (Alg. 4).
    threads > 1 splits the columns over host threads (same result bit for bit)."""
    lib = _load()
    N = len(dims)
    dims_a = np.asarray(dims, dtype=np.int64)
    ranks_a = np.asarray(ranks, dtype=np.int32)
    coords = _u32(coords)
    vals = _f64(vals)
    nnz = vals.shape[0]
    Us = [_f64(U[m]) if U[m] is not None else np.zeros((dims[m], ranks[m])) for m in range(N)]
    P = int(np.prod([ranks[m] for m in range(N) if m != mode], dtype=np.int64))
    Y = np.zeros((dims[mode], P), dtype=np.float64)
    args = (N, _ptr(dims_a, ctypes.c_int64), _ptr(ranks_a, ctypes.c_int), nnz, _ptr(coords, ctypes.c_uint32),
            _ptr(vals, ctypes.c_double), mode, _ptr_array(Us), _ptr(Y, ctypes.c_double))
    if threads > 1:
        lib.orc_ttmc_par(*args, int(threads))
    else:
        lib.orc_ttmc(*args)
    return Y


def kron_count() -> int:
    return int(_load().orc_kron_count())


def kron_reset() -> None:
    _load().orc_kron_reset()


# --------------------------------------------------------------------------- QRP
@dataclass
class QRPResult:
    Q: np.ndarray      # m x k, orthonormal columns
    piv: np.ndarray    # k original column indices, in pivot order
    rdiag: np.ndarray  # k diagonal entries of R


def qrp(A, k, threads=1):
    """Householder QR with column pivoting truncated at k reflectors (Section III-D)."""
    lib = _load()
    A = _f64(A)
    m, n = A.shape
    Q = np.zeros((m, k), dtype=np.float64)
    piv = np.zeros(k, dtype=np.int64)
    rdiag = np.zeros(k, dtype=np.float64)
    args = (_ptr(A, ctypes.c_double), m, n, n, k, _ptr(Q, ctypes.c_double), _ptr(piv, ctypes.c_int64),
            _ptr(rdiag, ctypes.c_double))
    rc = lib.orc_qrp_par(*args, int(threads)) if threads > 1 else lib.orc_qrp(*args)
    if rc != 0:
        raise ValueError(f"qrp: k={k} exceeds min(m={m}, n={n})")
    return QRPResult(Q, piv, rdiag)


def gram(Y, threads=1):
    """Y Y^T (Section III-D, fat case)."""
    lib = _load()
    Y = _f64(Y)
    m, n = Y.shape
    S = np.zeros((m, m), dtype=np.float64)
    if threads > 1:
        lib.orc_gram_par(_ptr(Y, ctypes.c_double), m, n, _ptr(S, ctypes.c_double), int(threads))
    else:
        lib.orc_gram(_ptr(Y, ctypes.c_double), m, n, _ptr(S, ctypes.c_double))
    return S


def qrp_factor(Y, R, direct=False, threads=1):
    """The factor update of Alg. 2: U_n = QRP(Y_(n), R_n).  When Y_(n) is fat
    (P_n > I_n) the paper runs QRP on Y Y^T; ``direct`` keeps QRP on Y itself."""
    m, n = Y.shape
    A = Y if (direct or n <= m) else gram(Y, threads)
    return qrp(A, R, threads)


# --------------------------------------------------------------------------- core
def core(Y_last, U_last, ranks, threads=1):
    """G = Y x_N U_N^T  <=>  G_(N) = U_N^T Y_(N)  (Section III-B).  Returns G with shape ranks."""
    lib = _load()
    Y = _f64(Y_last)
    U = _f64(U_last)
    I_N, P = Y.shape
    R_N = U.shape[1]
    G = np.zeros(P * R_N, dtype=np.float64)
    args = (I_N, P, R_N, _ptr(Y, ctypes.c_double), _ptr(U, ctypes.c_double), _ptr(G, ctypes.c_double))
    if threads > 1:
        lib.orc_core_par(*args, int(threads))
    else:
        lib.orc_core(*args)
    return G.reshape(tuple(ranks))


def fit_from_core(normX2: float, G) -> float:
    """1 - ||X - [[G; U]]|| / ||X|| written through ||G|| (valid for orthonormal U)."""
    g2 = float(np.sum(np.asarray(G, dtype=np.float64) ** 2))
    return 1.0 - np.sqrt(max(0.0, normX2 - g2)) / np.sqrt(normX2)


# --------------------------------------------------------------------------- HOOI
@dataclass
class HOOIResult:
    U: list
    G: np.ndarray
    fits: list
    pivots: list       # per sweep, per mode: pivot columns chosen by QRP (None in SVD mode)
    rdiags: list


def hooi(dims, ranks, coords, vals, U0, iters, direct=False, svd=False, coalesced=False, threads=1):
    """Algorithm 2: sparse Tucker by HOOI with QRP (or SVD, Alg. 1, as a check).

    U0: list of initial factors (I_m x R_m); U0[0] is never read (mode 1 is the first
    factor updated).  Returns the factors, the core and the fit after every sweep.
    threads > 1 runs the column-split routines (same results bit for bit)."""
    N = len(dims)
    if not coalesced:
        coords, vals = coalesce(coords, vals)
    nx2 = norm2(vals)
    U = [None] + [_f64(U0[m]) for m in range(1, N)]
    fits, pivots, rdiags = [], [], []
    Y = None
    for _ in range(iters):
        pv, rd = [], []
        for n in range(N):
            Y = ttmc(dims, ranks, coords, vals, n, U, threads)
            if svd:
                Ul, _, _ = np.linalg.svd(Y, full_matrices=False)
                U[n] = Ul[:, : ranks[n]].copy()
                pv.append(None)
                rd.append(None)
            else:
                res = qrp_factor(Y, ranks[n], direct=direct, threads=threads)
                U[n] = res.Q
                pv.append(res.piv)
                rd.append(res.rdiag)
        G = core(Y, U[N - 1], ranks, threads)
        fits.append(fit_from_core(nx2, G))
        pivots.append(pv)
        rdiags.append(rd)
    return HOOIResult(U, G, fits, pivots, rdiags)


# --------------------------------------------------------------------------- adjoint
def loss_grad(dims, ranks, coords, vals, U, G):
    """L = 1/2 sum_z (xhat_z - x_z)^2 with xhat = [[G; U_1..U_N]] at the observed
    coordinates, and dL/dU_m, dL/dG.  Plain FP64 loops (no coalescing: each listed
    entry is one observation)."""
    lib = _load()
    N = len(dims)
    dims_a = np.asarray(dims, dtype=np.int64)
    ranks_a = np.asarray(ranks, dtype=np.int32)
    coords = _u32(coords)
    vals = _f64(vals)
    nnz = vals.shape[0]
    Us = [_f64(u) for u in U]
    Gf = _f64(G).reshape(-1)
    dU = [np.zeros((dims[m], ranks[m]), dtype=np.float64) for m in range(N)]
    dG = np.zeros(Gf.shape[0], dtype=np.float64)
    loss = ctypes.c_double(0.0)
    lib.orc_loss_grad(N, _ptr(dims_a, ctypes.c_int64), _ptr(ranks_a, ctypes.c_int), nnz,
                      _ptr(coords, ctypes.c_uint32), _ptr(vals, ctypes.c_double), _ptr_array(Us),
                      _ptr(Gf, ctypes.c_double), ctypes.byref(loss), _ptr_array(dU), _ptr(dG, ctypes.c_double))
    return loss.value, dU, dG.reshape(tuple(ranks))
