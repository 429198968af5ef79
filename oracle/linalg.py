"""ctypes wrappers around the oracle's C routines (oracle/linalg.c).

Test infrastructure only.  FP64 throughout.  Nothing here is shared with the
CUDA library.
"""
import ctypes
import threading

import numpy as np

from . import _build

_lib = None
_lib_lock = threading.Lock()


def _L():
    global _lib
    if _lib is not None:
        return _lib
    with _lib_lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        lib.orc_cholesky.argtypes = [ctypes.c_int, dp, dp]
        lib.orc_cholesky.restype = ctypes.c_int
        lib.orc_forward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_backward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.orc_jacobi.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_double]
        lib.orc_jacobi.restype = ctypes.c_int
        lib.orc_ldlt_negative_count.argtypes = [ctypes.c_int, dp]
        lib.orc_ldlt_negative_count.restype = ctypes.c_int
        lib.orc_band_cholesky.argtypes = [ctypes.c_int, ctypes.c_int, dp]
        lib.orc_band_cholesky.restype = ctypes.c_int
        lib.orc_band_solve.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, dp]
        lib.orc_band_solve.restype = None
        lib.orc_band_negative_count.argtypes = [ctypes.c_int, ctypes.c_int, dp]
        lib.orc_band_negative_count.restype = ctypes.c_int
        ip = ctypes.POINTER(ctypes.c_int)
        lib.orc_ldlt_null.argtypes = [ctypes.c_int, dp, ctypes.c_double, dp, dp, ip]
        lib.orc_ldlt_null.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


class NotSPDError(ValueError):
    def __init__(self, pivot):
        super().__init__("matrix is not positive definite (pivot %d)" % pivot)
        self.pivot = pivot


def cholesky(A):
    """Lower-triangular L with A = L L^T (dense, textbook algorithm)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    info = _L().orc_cholesky(n, _p(A), _p(L))
    if info:
        raise NotSPDError(info - 1)
    return L


def forward(L, B):
    """Solve L X = B (L lower triangular)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(L.shape[0], -1), dtype=np.float64).copy()
    _L().orc_forward(L.shape[0], X.shape[1], _p(L), _p(X))
    return X[:, 0] if vec else X


def backward(L, B):
    """Solve L^T X = B (L lower triangular)."""
    L = np.ascontiguousarray(L, dtype=np.float64)
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(L.shape[0], -1), dtype=np.float64).copy()
    _L().orc_backward(L.shape[0], X.shape[1], _p(L), _p(X))
    return X[:, 0] if vec else X


def cho_solve(L, B):
    """Solve (L L^T) X = B."""
    return backward(L, forward(L, B))


def jacobi_eigh(S, tol=1e-15, max_sweeps=60):
    """All eigenpairs of the symmetric matrix S by the cyclic Jacobi method.

    Returns (w, V) with w ascending and S = V diag(w) V^T.
    """
    S = np.array(S, dtype=np.float64, order="C", copy=True)
    S = 0.5 * (S + S.T)
    n = S.shape[0]
    if n == 0:
        return np.zeros(0), np.zeros((0, 0))
    w = np.zeros(n)
    V = np.zeros((n, n))
    sweeps = _L().orc_jacobi(n, _p(S), _p(w), _p(V), max_sweeps, tol)
    if sweeps < 0:
        raise RuntimeError("Jacobi did not converge in %d sweeps" % max_sweeps)
    order = np.argsort(w, kind="stable")
    return w[order], V[:, order]


def negative_count(A):
    """Number of negative eigenvalues of symmetric A via LDL^T (Sylvester's law)."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    A = 0.5 * (A + A.T)
    k = _L().orc_ldlt_negative_count(A.shape[0], _p(A))
    if k < 0:
        raise RuntimeError("LDL^T met a zero pivot")
    return k


# ---- band matrices (method mode): lower band, row-major by rows, entry
# (i, j), i - b <= j <= i, at AB[i, j - i + b]

def half_bandwidth(A):
    """Largest |i - j| over the nonzero entries of a dense or sparse matrix."""
    if hasattr(A, "tocoo"):
        c = A.tocoo()
        r, k = c.row[c.data != 0], c.col[c.data != 0]
    else:
        r, k = np.nonzero(A)
    return int(np.abs(r - k).max()) if len(r) else 0


def to_band(A, b):
    """Lower band (n x (b+1)) of the symmetric matrix A (dense or sparse)."""
    n = A.shape[0]
    AB = np.zeros((n, b + 1))
    if hasattr(A, "tocoo"):
        c = A.tocoo()
        low = c.row >= c.col
        r, k, v = c.row[low], c.col[low], c.data[low]
        if np.any(r - k > b):
            raise ValueError("entry outside the band")
        np.add.at(AB, (r, k - r + b), v)
    else:
        for d in range(b + 1):
            AB[d:, b - d] = np.diagonal(A, -d)
    return AB


def band_cholesky(AB):
    """Band factor L (same storage) with A = L L^T."""
    L = np.ascontiguousarray(AB, dtype=np.float64).copy()
    info = _L().orc_band_cholesky(L.shape[0], L.shape[1] - 1, _p(L))
    if info:
        raise NotSPDError(info - 1)
    return L


def band_solve(LB, B):
    """Solve (L L^T) X = B with a band factor from band_cholesky."""
    LB = np.ascontiguousarray(LB, dtype=np.float64)
    vec = B.ndim == 1
    X = np.ascontiguousarray(B.reshape(LB.shape[0], -1), dtype=np.float64).copy()
    _L().orc_band_solve(LB.shape[0], LB.shape[1] - 1, _p(LB), X.shape[1], _p(X))
    return X[:, 0] if vec else X


def band_negative_count(AB):
    """Number of negative eigenvalues of a symmetric band matrix (LDL^T inertia)."""
    AB = np.ascontiguousarray(AB, dtype=np.float64)
    k = _L().orc_band_negative_count(AB.shape[0], AB.shape[1] - 1, _p(AB))
    if k < 0:
        raise RuntimeError("band LDL^T met a zero pivot")
    return k


def ldlt_null(K, tau):
    """Regularised LDL^T of symmetric positive semi-definite K in the given
    order (linalg.c: orc_ldlt_null): returns (L unit lower, d, null flags);
    pivots with d_k <= tau K_kk are null (d_k = 0, column k of L zero)."""
    K = np.ascontiguousarray(0.5 * (K + K.T), dtype=np.float64)
    n = K.shape[0]
    L = np.zeros_like(K)
    d = np.zeros(n)
    null = np.zeros(n, dtype=np.int32)
    r = _L().orc_ldlt_null(n, _p(K), float(tau), _p(L), _p(d),
                           null.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    if r < 0:
        raise MemoryError("orc_ldlt_null")
    return L, d, null.astype(bool)
