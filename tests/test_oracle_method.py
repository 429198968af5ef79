"""Pins of the oracle's multilevel preconditioner and CG (Sections 2.1, 3.1, 3.2, 5).

Expected values come from the paper's theorems (Lemma upper_bound, Theorem
multilevelrate with Lemma spectral1's C_1 = 1/eta), from exact special cases
(one subdomain covering the domain), from a direct sparse solve, and from the
behaviour the paper reports (iterations flat in the contrast, Tab. 1 and 3).
The CG Lanczos estimate of the spectrum of BA is pinned by exact
termination on a diagonal system with a known spectrum.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic_inputs as si
from oracle import fem, method


def _explicit(H):
    n = H.n
    I = np.eye(n)
    Bm = np.stack([H.apply_preconditioner(I[:, j]) for j in range(n)], axis=1)
    return Bm


@pytest.mark.parametrize("levels", [2, 3])
def test_preconditioner_spd_and_condition_bounds(levels):
    mesh = fem.Mesh((16, 16), 0b1)
    kap = si.channels_2d(16, 3, 1e4, seed=1)
    eta = 0.3
    H = method.Hierarchy(mesh, kap, (4, 4), 1, levels, (2, 2), 10 ** 6, eta)
    Bm = _explicit(H)
    assert np.allclose(Bm, Bm.T, atol=1e-10 * np.abs(Bm).max())
    assert np.linalg.eigvalsh(0.5 * (Bm + Bm.T)).min() > 0
    A = H.A.toarray()
    # eigenvalues of BA = those of A^{1/2} B A^{1/2}
    Ls = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(Ls.T @ Bm @ Ls)
    L = levels - 1
    k0 = 4                                       # 2D box colouring, also a0 = b0 = k0
    C1 = 1.0 / eta                               # Lemma spectral1, b^1
    C = 2 * (1 + k0 * k0 * C1)
    lower = 1.0 / (C ** L * (1 + k0 * C1 / (C - 1)))
    assert ev.max() <= 1 + k0 * L + 1e-9         # Lemma upper_bound
    assert ev.min() >= lower                     # Theorem multilevelrate (lower half)


def test_one_subdomain_covering_domain():
    """B = A^{-1} + P0 A0^{-1} P0^T: BA has eigenvalues in {1, 2}; CG needs <= 2 steps."""
    mesh = fem.Mesh((12, 12), 0b1)
    kap = si.channels_2d(12, 2, 1e3, seed=0)
    b = fem.load_vector(mesh)
    H = method.Hierarchy(mesh, kap, (1, 1), 1, 2, (1, 1), 3, 2.0)
    assert H.n0 == 3
    x, it, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-12)
    assert it <= 2
    H1 = method.Hierarchy(mesh, kap, (1, 1), 1, 2, (1, 1), 3, 0.3)
    assert H1.n0 == 0                            # all lambda = 1 when chi = 1
    x, it, *_ = method.pcg(H1.A, b, H1.apply_preconditioner, 1e-12)
    assert it == 1


def test_galerkin_and_coarse_matrices():
    mesh = fem.Mesh((32, 32), 0b1)
    kap = si.channels_2d(32, 4, 1e6, seed=2)
    H = method.Hierarchy(mesh, kap, (4, 4), 2, 3, (2, 2), 8, 0.3)
    lev1 = H.levels[1]
    P = lev1.P.toarray()
    assert np.allclose(lev1.A_level, P.T @ H.A.toarray() @ P, atol=1e-9)
    assert np.linalg.eigvalsh(lev1.A_level).min() > 0
    assert np.linalg.eigvalsh(H.A0).min() > 0
    # fine basis functions are b-normalised: a(phi, phi) = 1 (diag of A_1)
    assert np.allclose(np.diag(lev1.A_level), 1.0, atol=1e-8)
    for s in lev1.subs:
        assert np.all(s["lam"] >= -1e-10)
        assert s["m"] <= 8


def test_solution_matches_direct_solve():
    w = si.channels64()
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    kap = w.coefficient()
    H = method.Hierarchy(mesh, kap, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta)
    b = fem.load_vector(mesh)
    x, it, hist, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-12)
    xd = spla.spsolve(H.A.tocsc(), b)
    err_A = np.sqrt((x - xd) @ (H.A @ (x - xd)) / (xd @ (H.A @ xd)))
    assert err_A < 1e-10
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) < 1e-8
    x8, it8, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-8)
    assert 20 <= it8 <= 60


def test_iterations_flat_in_contrast_one_level_not():
    """Spectral coarse space: #IT flat as the channel contrast grows (Tab. 1, 3 pattern);
    one-level Schwarz (no coarse space) needs far more iterations."""
    mesh = fem.Mesh((64, 64), 0b1)
    b = fem.load_vector(mesh)
    two, one = [], []
    for c in (1e2, 1e4, 1e6):
        kap = si.channels_2d(64, 8, c, seed=0)
        H = method.Hierarchy(mesh, kap, (8, 8), 2, 2, (2, 2), 8, 0.3)
        two.append(method.pcg(H.A, b, H.apply_preconditioner, 1e-8)[1])
        one.append(method.pcg(H.A, b, H.apply_one_level, 1e-8, maxit=3000)[1])
    assert max(two) - min(two) <= 5
    assert max(one) > 1.5 * max(two)


def test_lanczos_condition_recovers_the_spectrum():
    """CG's Lanczos tridiagonal (built from the recorded alphas and betas):
    with A = diag(d) and B = diag(1/w), BA has the eigenvalues d/w; from a
    right-hand side touching all 12 of them, CG ends after 12 steps and the
    extreme eigenvalues of the tridiagonal are the extreme d/w (exact
    termination); after fewer steps its eigenvalues lie inside them
    (interlacing)."""
    d = np.arange(1.0, 13.0) ** 2
    w = np.linspace(0.5, 2.0, 12)
    ev = np.sort(d / w)
    A = np.diag(d)
    b = np.ones(12)
    _, it, _, al, be = method.pcg(A, b, lambda r: r / w, 1e-12, maxit=40)
    assert it == 12
    lo, hi = method.lanczos_condition(al, be)
    assert abs(lo - ev[0]) <= 1e-8 * ev[0] and abs(hi - ev[-1]) <= 1e-8 * ev[-1]
    _, it5, _, al5, be5 = method.pcg(A, b, lambda r: r / w, 1e-12, maxit=5)
    assert it5 == 5
    lo5, hi5 = method.lanczos_condition(al5, be5)
    assert ev[0] - 1e-9 <= lo5 < hi5 <= ev[-1] + 1e-9 and hi5 < ev[-1]
