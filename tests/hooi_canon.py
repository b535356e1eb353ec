"""Sign-fixed views of a Tucker model, shared by the stored-result script and the GPU tests.

QRP fixes each factor column's sign through the Householder convention, so an FP32 path
and the FP64 oracle that choose the same pivots produce the same columns; comparing them
elementwise across a stored file still needs one convention that both sides apply to
their own factors.  Here every column is flipped so that its largest-magnitude entry is
positive, and the core's slices are flipped with it (the model [[G; U_1..U_N]] is
unchanged).  No arithmetic of the method lives here."""
import numpy as np

SKETCH_COLS = 4


def column_signs(U):
    """+1 / -1 per column: the sign of the column's largest-magnitude entry."""
    U = np.asarray(U, dtype=np.float64)
    i = np.argmax(np.abs(U), axis=0)
    return np.where(U[i, np.arange(U.shape[1])] < 0, -1.0, 1.0)


def canonical(U, G):
    """Factors and core with every factor column's sign fixed."""
    Uc, Gc = [], np.array(G, dtype=np.float64)
    for n, u in enumerate(U):
        s = column_signs(u)
        Uc.append(np.asarray(u, dtype=np.float64) * s)
        shape = [1] * Gc.ndim
        shape[n] = -1
        Gc = Gc * s.reshape(shape)
    return Uc, Gc


def sketch(U, n):
    """U^T W_n with W_n of seeded N(0, 1) entries (numpy default_rng(7 + n)): R_n x 4 numbers
    that fingerprint the factor itself (columns, order and signs)."""
    W = np.random.default_rng(7 + n).standard_normal((U.shape[0], SKETCH_COLS))
    return np.asarray(U, dtype=np.float64).T @ W
