"""Pins of the oracle's LAPACK-free dense Cholesky and Jacobi eigensolver.

Closed forms (the discrete Laplacian's spectrum) and library routines used as
independent brute force (numpy's LAPACK, called here in the test only).
"""
import numpy as np
import pytest

from oracle import linalg


def test_jacobi_tridiagonal_closed_form():
    # T = tridiag(-1, 2, -1) of order n: eigenvalues 2 - 2 cos(k pi / (n+1)),
    # eigenvectors sin(j k pi / (n+1))
    n = 37
    T = 2 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    w, V = linalg.jacobi_eigh(T)
    k = np.arange(1, n + 1)
    assert np.allclose(w, 2 - 2 * np.cos(k * np.pi / (n + 1)), atol=1e-13)
    v1 = np.sin(np.arange(1, n + 1) * np.pi / (n + 1))
    v1 /= np.linalg.norm(v1)
    assert abs(abs(V[:, 0] @ v1) - 1) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 9, 60])
def test_jacobi_matches_lapack(n):
    rng = np.random.default_rng(n)
    M = rng.standard_normal((n, n))
    S = M + M.T
    w, V = linalg.jacobi_eigh(S)
    assert np.allclose(w, np.linalg.eigvalsh(S), atol=1e-12 * max(1, np.abs(w).max()))
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.allclose(V @ np.diag(w) @ V.T, S, atol=1e-11 * max(1, np.abs(S).max()))


def test_jacobi_semidefinite_kernel():
    rng = np.random.default_rng(3)
    X = rng.standard_normal((20, 5))
    w, V = linalg.jacobi_eigh(X @ X.T)
    assert np.sum(np.abs(w) < 1e-10) == 15


def test_cholesky_and_solves_match_lapack():
    rng = np.random.default_rng(7)
    M = rng.standard_normal((40, 40))
    A = M @ M.T + 40 * np.eye(40)
    L = linalg.cholesky(A)
    assert np.allclose(L, np.linalg.cholesky(A), atol=1e-12)
    B = rng.standard_normal((40, 3))
    assert np.allclose(linalg.cho_solve(L, B), np.linalg.solve(A, B), atol=1e-12)
    assert np.allclose(linalg.forward(L, B), np.linalg.solve(L, B), atol=1e-12)
    assert np.allclose(linalg.backward(L, B), np.linalg.solve(L.T, B), atol=1e-12)


def test_cholesky_reports_failing_pivot():
    A = np.diag([1.0, 2.0, -1.0, 4.0])
    with pytest.raises(linalg.NotSPDError) as e:
        linalg.cholesky(A)
    assert e.value.pivot == 2


def test_negative_count_matches_spectrum():
    rng = np.random.default_rng(11)
    M = rng.standard_normal((30, 30))
    S = M + M.T
    assert linalg.negative_count(S) == int(np.sum(np.linalg.eigvalsh(S) < 0))
    T = 2 * np.eye(20) - np.eye(20, k=1) - np.eye(20, k=-1)
    k = np.arange(1, 21)
    ev = 2 - 2 * np.cos(k * np.pi / 21)
    assert linalg.negative_count(T - 1.05 * np.eye(20)) == int(np.sum(ev < 1.05))
