"""Pins of the oracle's local generalized eigenproblems (Section 3.3, 3.4, 4.2).

Invariants the paper proves (spectrum structure, kernels, projection
stability), and brute force via scipy's LAPACK-based symmetric-definite
solver on the spectrally transformed pencil (test-only).
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic_inputs as si
from oracle import decomposition as dd
from oracle import fem, method


def _local(mesh, kap, parts, overlap, i):
    dec = dd.Decomposition(mesh, parts, overlap, 2, (2,) * mesh.dim)
    chis, _ = dec.partition_of_unity()
    s = dec.fine[i]
    nn = s.neumann_nodes()
    Abar = fem.assemble_neumann(mesh, kap, s.element_mask)[nn][:, nn].toarray()
    chi = chis[i]
    return Abar, chi[:, None] * Abar * chi[None, :], chi


@pytest.fixture(scope="module")
def channel_problem():
    mesh = fem.Mesh((24, 24), 0b1)
    kap = si.channels_2d(24, 4, 1e6, seed=3)
    return mesh, kap


def test_floating_subdomain_kernel_is_constants(channel_problem):
    """Lemma (Section 3.4): ker abar = constants for a floating subdomain; lambda_1 = 0 simple."""
    mesh, kap = channel_problem
    Abar, B, chi = _local(mesh, kap, (3, 3), 2, 4)       # centre subdomain, floating
    lam, W = method.gevp(Abar, B, rank_reveal=False)
    assert abs(lam[0]) < 1e-9 and lam[1] > 1e-9
    w0 = W[:, 0] / W[np.argmax(np.abs(W[:, 0])), 0]
    assert np.allclose(w0, 1.0, atol=1e-6)


def test_dirichlet_subdomain_has_positive_spectrum(channel_problem):
    mesh, kap = channel_problem
    Abar, B, chi = _local(mesh, kap, (3, 3), 2, 0)       # touches x = 0
    lam, W = method.gevp(Abar, B, rank_reveal=False)
    assert lam[0] > 1e-8


def test_spectrum_structure_and_orthogonality(channel_problem):
    """#(lambda = inf) = dim ker B = #(chi = 0); B-orthonormal, Abar-orthogonal, residuals."""
    mesh, kap = channel_problem
    Abar, B, chi = _local(mesh, kap, (3, 3), 2, 4)
    lam, W = method.gevp(Abar, B, rank_reveal=False)
    n = Abar.shape[0]
    assert n - len(lam) == int(np.sum(chi == 0.0))
    assert np.all(np.diff(lam) >= -1e-12 * np.abs(lam).max())
    assert np.allclose(W.T @ B @ W, np.eye(len(lam)), atol=1e-8)
    G = W.T @ Abar @ W
    assert np.allclose(G, np.diag(lam), atol=1e-7 * max(1.0, lam.max()))
    R = Abar @ W - (B @ W) * lam[None, :]
    scale = np.abs(Abar).sum(axis=1).max() * np.abs(W).max(axis=0)   # ||Abar||_inf ||w||_inf
    assert (np.abs(R).max(axis=0) / scale).max() < 1e-10


def test_matches_lapack_on_transformed_pencil(channel_problem):
    """Brute force: eigvals of B x = mu (Abar + B) x via scipy, lambda = 1/mu - 1."""
    mesh, kap = channel_problem
    Abar, B, chi = _local(mesh, kap, (3, 3), 2, 5)
    lam, W = method.gevp(Abar, B, rank_reveal=False)
    mu = sla.eigh(B, Abar + B, eigvals_only=True)
    mu = np.sort(mu)[::-1]
    lam_ref = 1.0 / mu[: len(lam)] - 1.0
    k = lam < 10.0
    assert np.allclose(lam[k], lam_ref[k], rtol=1e-7, atol=1e-9)


def test_projection_stability(channel_problem):
    """Eq. a_stability and ba_stability (Lemma in Section 3.3) on random vectors."""
    mesh, kap = channel_problem
    Abar, B, chi = _local(mesh, kap, (3, 3), 2, 4)
    lam, W = method.gevp(Abar, B, rank_reveal=False)
    rng = np.random.default_rng(0)
    r = 1                                             # dim ker abar (floating)
    for m in (1, 3, 6):
        assert m >= r
        for _ in range(5):
            v = rng.standard_normal(Abar.shape[0])
            Pv = W[:, :m] @ (W[:, :m].T @ (B @ v))
            a = lambda u: u @ Abar @ u
            b = lambda u: u @ B @ u
            assert a(Pv) <= a(v) * (1 + 1e-9) + 1e-9
            assert a(v - Pv) <= a(v) * (1 + 1e-9) + 1e-9
            assert b(v - Pv) <= a(v - Pv) / lam[m] * (1 + 1e-7) + 1e-9


def test_rank_revealing_drops_common_kernel():
    """Generating system with exact duplicates (Section 4.2): same finite spectrum."""
    rng = np.random.default_rng(5)
    n = 12
    M = rng.standard_normal((n, n))
    Abar = M @ M.T
    x = np.r_[np.ones(6), np.zeros(6)]
    B = x[:, None] * Abar * x[None, :]
    lam, _ = method.gevp(Abar, B, rank_reveal=False)
    # duplicate two generators (columns of the basis) -> singular pencil
    G = np.eye(n)[:, list(range(n)) + [7, 9]]
    A2 = G.T @ Abar @ G
    x2 = np.r_[x, 0, 0]
    B2 = x2[:, None] * A2 * x2[None, :]
    lam2, W2 = method.gevp(A2, B2, rank_reveal=True)
    assert np.allclose(lam2, lam, rtol=1e-8)
    assert np.allclose(W2.T @ B2 @ W2, np.eye(len(lam2)), atol=1e-8)


def test_selection_rule():
    lam = np.array([0.0, 0.1, 0.29999, 0.3, 0.5])
    assert method.select_count(lam, 8, 0.3) == 3                # strict lambda < eta
    assert method.select_count(lam, 2, 0.3) == 2                # cap nev_max


def test_sylvester_count_matches_eigenvalue_count(channel_problem):
    """#negative eigenvalues of (Abar - theta B) = #{lambda < theta} (congruence with (Abar+B)^{-1/2})."""
    from oracle import linalg
    mesh, kap = channel_problem
    for i in (0, 4, 7):
        Abar, B, chi = _local(mesh, kap, (3, 3), 2, i)
        lam, _ = method.gevp(Abar, B, rank_reveal=False)
        for theta in (0.05, 0.3, 1.7):
            assert linalg.negative_count(Abar - theta * B) == int(np.sum(lam < theta))
