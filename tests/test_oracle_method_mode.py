"""Pins of the oracle's method mode (band factors and subspace iteration on
the fine level) against the dense oracle and against brute force.

  * band Cholesky, band solves and the band LDL^T inertia count against the
    dense textbook routines and numpy's eigvalsh (brute force);
  * block subspace iteration with Rayleigh-Ritz (Section 4.2's shift-invert
    eigensolver replaced by the plain algorithm) against the complete
    dense GEVP solution: eigenvalues, b-orthonormality, residuals;
  * the whole method-mode hierarchy against the dense oracle on the 64 x 64
    channel workload (two levels), a three-level case and a 3D case (8^3
    elements, 2^3 subdomains, layered kappa 1 / 1e4): selected counts
    and coarse dimensions exact, eigenvalues to 1e-8 relative (1e-7 on the
    middle level), the preconditioner application and the PCG iterates to
    1e-8;
  * worker processes give the same result as the in-process loop;
  * the bounded fine-level sample (the host baseline of the 3D workloads)
    against the dense oracle's eigenvalues and counts on sampled subdomains.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import fem, linalg, method, method_mode


def _band_spd(n, b, rng, shift=1.0):
    M = rng.standard_normal((n, n))
    band = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= b
    S = np.where(band, M + M.T, 0.0)
    return S + np.diag(np.abs(S).sum(axis=1) + shift)


@pytest.mark.parametrize("n,b", [(1, 0), (7, 3), (40, 1), (65, 12), (90, 89)])
def test_band_routines_match_dense(n, b):
    rng = np.random.default_rng(n + b)
    S = _band_spd(n, b, rng)
    assert linalg.half_bandwidth(S) == min(b, n - 1)
    AB = linalg.to_band(S, b)
    L = linalg.band_cholesky(AB)
    Ld = linalg.cholesky(S)
    for d in range(b + 1):
        assert np.allclose(L[d:, b - d], np.diagonal(Ld, -d), rtol=0, atol=1e-12 * np.abs(Ld).max())
    X = rng.standard_normal((n, 3))
    Y = linalg.band_solve(L, X)
    assert np.abs(S @ Y - X).max() <= 1e-10 * np.abs(X).max()
    # inertia of S - t I for shifts between eigenvalues
    ev = np.linalg.eigvalsh(S)
    for t in (ev[0] - 1.0, 0.5 * (ev[0] + ev[-1]), ev[-1] + 1.0):
        if np.min(np.abs(ev - t)) > 1e-6:
            assert linalg.band_negative_count(linalg.to_band(S - t * np.eye(n), b)) == int(np.sum(ev < t))


def test_band_cholesky_reports_the_failing_pivot():
    S = np.diag([1.0, 2.0, -1.0, 4.0])
    with pytest.raises(linalg.NotSPDError) as e:
        linalg.band_cholesky(linalg.to_band(S, 1))
    assert e.value.pivot == 2


def test_subspace_iteration_matches_dense_gevp():
    mesh = fem.Mesh((24, 24), 0b1)
    kap = si.channels_2d(24, 4, 1e6, seed=3)
    dec = method.Decomposition(mesh, (3, 3), 2, 2, (1, 1))
    chis, _ = dec.partition_of_unity()
    Ke = fem.element_matrices(mesh, kap)
    en = mesh.element_nodes()
    for i in (0, 4):                                   # touching x = 0, floating
        s = dec.fine[i]
        nn = s.neumann_nodes()
        Abar = method_mode.local_neumann(Ke, en, s.element_mask, nn, mesh.num_nodes)
        _, Ad, Bd = method.fine_pencil(mesh, Ke, en, s, chis[i])
        assert np.abs(Abar.toarray() - Ad).max() <= 1e-12 * np.abs(Ad).max()
        B = chis[i][:, None] * Abar.toarray() * chis[i][None, :]
        K = Abar.toarray() + 1e-2 * B
        KL = linalg.band_cholesky(linalg.to_band(K, linalg.half_bandwidth(K)))
        theta, X, its = method_mode.subspace_iteration(Abar.toarray(), B, KL, 6, 0.3, 14, 1e-8, 500,
                                                       np.random.default_rng(1))
        assert its > 0
        lam, _ = method.gevp(Ad, Bd, rank_reveal=False)
        m = method.select_count(theta, 6, 0.3)
        assert m == method.select_count(lam, 6, 0.3)
        err = np.abs(theta[:m] - lam[:m]) / np.maximum(np.abs(lam[:m]), 1e-4)
        assert err.max() < 1e-9, err
        assert theta[m] >= lam[m] - 1e-12 and theta[m] > 0.3      # Ritz values bound from above
        assert np.allclose(X.T @ B @ X, np.eye(X.shape[1]), atol=1e-9)


CASES = {
    "channels64": lambda: (si.channels64(), None),
    "three_level": lambda: (None, dict(n=(32, 32), parts=(4, 4), overlap=2, levels=3, group=(2, 2), nev=6,
                                       eta=0.3, kappa=si.channels_2d(32, 4, 1e5, seed=5))),
    "three_d": lambda: (None, dict(n=(8, 8, 8), parts=(2, 2, 2), overlap=1, levels=2, group=(1, 1, 1), nev=6,
                                   eta=0.3, kappa=si.layered_3d(8, seed=3))),
}


def _pair(name, processes=1):
    w, c = CASES[name]()
    if w is not None:
        c = dict(n=w.n, parts=w.parts, overlap=w.overlap, levels=w.levels, group=w.group, nev=w.nev_max,
                 eta=w.eta, kappa=w.coefficient())
    mesh = fem.Mesh(c["n"], 0b1)
    args = (mesh, c["kappa"], c["parts"], c["overlap"], c["levels"], c["group"], c["nev"], c["eta"])
    return c, mesh, method.Hierarchy(*args), method_mode.MethodModeHierarchy(*args, tol=1e-10, processes=processes)


@pytest.mark.parametrize("name", ["channels64", "three_level", "three_d"])
def test_method_mode_matches_dense_oracle(name):
    c, mesh, D, M = _pair(name)
    for l in range(D.L, 0, -1):
        for a, b in zip(D.levels[l].subs, M.levels[l].subs):
            assert a["m"] == b["m"]
            k = a["m"]
            if k == 0:                               # nothing below eta here
                continue
            err = np.abs(a["lam"][:k] - b["lam"][:k]) / np.maximum(np.abs(a["lam"][:k]), 1e-3 * c["eta"])
            # middle level: its pencil is built from the fine eigenvectors,
            # whose errors (residual 1e-10 over the gaps) enter at first order
            assert err.max() < (1e-8 if l == D.L else 1e-7), (l, err)
    assert D.coarse_dims() == M.coarse_dims()
    rng = np.random.default_rng(2)
    r = rng.standard_normal(D.n)
    zd, zm = D.apply_preconditioner(r), M.apply_preconditioner(r)
    assert np.linalg.norm(zd - zm) <= 1e-8 * np.linalg.norm(zd)
    b = fem.load_vector(mesh)
    xd, itd, *_ = method.pcg(D.A, b, D.apply_preconditioner, 1e-8)
    xm, itm, *_ = method.pcg(M.A, b, M.apply_preconditioner, 1e-8)
    assert itd == itm
    assert np.linalg.norm(xd - xm) <= 1e-8 * np.linalg.norm(xd)


def test_worker_processes_give_the_same_hierarchy():
    w = si.channels64()
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    args = (mesh, w.coefficient(), w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta)
    M1 = method_mode.MethodModeHierarchy(*args, processes=1)
    M2 = method_mode.MethodModeHierarchy(*args, processes=2)
    for a, b in zip(M1.levels[M1.L].subs, M2.levels[M2.L].subs):
        assert np.array_equal(a["lam"], b["lam"]) and np.array_equal(a["W"], b["W"])
    assert np.array_equal(M1.A0, M2.A0)


def test_fine_level_sample_matches_dense_oracle():
    """The bounded fine-level sample that stands in for a full step on
    workloads too large for the host: its Ritz values and selected counts on
    sampled subdomains equal the dense oracle's complete GEVP solution."""
    c = CASES["three_d"]()[1]
    mesh = fem.Mesh(c["n"], 0b1)
    D = method.Hierarchy(mesh, c["kappa"], c["parts"], c["overlap"], c["levels"], c["group"], c["nev"], c["eta"])
    sample = [0, 3, 7]
    got = method_mode.fine_level_sample(c["n"], 0b1, c["kappa"], c["parts"], c["overlap"], c["levels"], c["group"],
                                        c["nev"], c["eta"], sample, processes=1, tol=1e-10)
    for i, g in zip(sample, got):
        ref = D.levels[D.L].subs[i]
        assert g["m"] == ref["m"] and g["eig_iterations"] > 0
        k = g["m"]
        err = np.abs(g["lam"][:k] - ref["lam"][:k]) / np.maximum(np.abs(ref["lam"][:k]), 1e-3 * c["eta"])
        assert k == 0 or err.max() < 1e-8, (i, err)
