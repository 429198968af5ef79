"""ctypes wrappers around the oracle's C routines (oracle/linalg.c).

Test infrastructure only.  FP64 throughout.  Nothing here is shared with the
CUDA library.
"""
import ctypes
import numpy as np

from . import _build

_lib = None


def _L():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(_build.build())
        dp = ctypes.POINTER(ctypes.c_double)
        _lib.orc_cholesky.argtypes = [ctypes.c_int, dp, dp]
        _lib.orc_cholesky.restype = ctypes.c_int
        _lib.orc_forward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.orc_backward.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        _lib.orc_jacobi.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_int, ctypes.c_double]
        _lib.orc_jacobi.restype = ctypes.c_int
        _lib.orc_ldlt_negative_count.argtypes = [ctypes.c_int, dp]
        _lib.orc_ldlt_negative_count.restype = ctypes.c_int
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
