"""Pins of the oracle's GEVP right-hand sides b^1, b^2, b^3 (Section 3.4,
Eq. cg_rhs_blf and original_geneo; Lemma spectral1).

* b^3 against b^1 through the identity abar(u, u) = b^1(u, u) + b^3(u, u)
  + 2 abar(chi u, (1 - chi) u) (a dropped term or sign in either fails it);
* b^2 against an element set built from the subdomain boxes geometrically
  (element e of subdomain i lies in the box of some j != i), assembled from
  the element matrices directly;
* b^2 <= b^1 in the Loewner order (b^1 - b^2 sums non-negative element forms);
* the kernel lemma of Section 3.4: for a subdomain away from the Dirichlet
  boundary the constant lies in ker abar but not in ker b^alpha;
* the fact used in the proof of Lemma spectral1: chi = 1 on every node of an
  element that belongs to no other subdomain;
* one subdomain covering the domain: no overlap, chi = 1, so b^2 = b^3 = 0;
* the condition bounds of Lemma upper_bound and Theorem multilevelrate with
  the constants C_1^2 = 1 + 1/eta and C_1^3 = 2 (1 + 1/eta) of Lemma spectral1.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import fem, method
from oracle.decomposition import Decomposition


def _setup(n=(12, 10), parts=(3, 2), overlap=1, seed=2):
    mesh = fem.Mesh(n, 0b1)
    kap = si.channels_2d(n[0], 2, 1e3, seed=seed)[: n[0] * n[1]]
    dec = Decomposition(mesh, parts, overlap, 2, (1, 1))
    chis, _ = dec.partition_of_unity()
    Ke = fem.element_matrices(mesh, kap)
    en = mesh.element_nodes()
    return mesh, kap, dec, chis, Ke, en


def test_b3_b1_identity():
    mesh, kap, dec, chis, Ke, en = _setup()
    rng = np.random.default_rng(0)
    for i, s in enumerate(dec.fine):
        nn, A, B1 = method.fine_pencil(mesh, Ke, en, s, chis[i], blf=1)
        _, A3, B3 = method.fine_pencil(mesh, Ke, en, s, chis[i], blf=3)
        assert np.array_equal(A, A3)
        chi = chis[i]
        for _ in range(3):
            u = rng.standard_normal(len(nn))
            lhs = u @ A @ u
            rhs = u @ B1 @ u + u @ B3 @ u + 2.0 * (chi * u) @ A @ ((1.0 - chi) * u)
            assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_b2_overlap_elements_from_box_geometry():
    mesh, kap, dec, chis, Ke, en = _setup()
    ovl = method.overlap_elements(dec)
    coords = mesh.element_coords()
    for i, s in enumerate(dec.fine):
        nn, A, B2 = method.fine_pencil(mesh, Ke, en, s, chis[i], blf=2, overlap_elements=ovl)
        pos = -np.ones(mesh.num_nodes, dtype=np.int64)
        pos[nn] = np.arange(len(nn))
        Aring = np.zeros_like(A)
        for e in range(mesh.num_elements):
            inside = lambda box: all(box[d][0] <= coords[e, d] < box[d][1] for d in range(mesh.dim))
            if not inside(s.ext):
                continue
            if not any(inside(t.ext) for j, t in enumerate(dec.fine) if j != i):
                continue
            loc = pos[en[e]]
            ok = loc >= 0
            Aring[np.ix_(loc[ok], loc[ok])] += Ke[e][np.ix_(ok, ok)]
        chi = chis[i]
        ref = chi[:, None] * Aring * chi[None, :]
        assert np.allclose(B2, ref, rtol=0, atol=1e-13 * np.abs(A).max())
        # b^2 <= b^1 (Loewner)
        _, _, B1 = method.fine_pencil(mesh, Ke, en, s, chis[i], blf=1)
        assert np.linalg.eigvalsh(B1 - B2).min() >= -1e-11 * np.abs(A).max()


def test_kernel_lemma_and_chi_on_interior_elements():
    mesh, kap, dec, chis, Ke, en = _setup(n=(16, 16), parts=(4, 4), overlap=2)
    ovl = method.overlap_elements(dec)
    floating = 0
    for i, s in enumerate(dec.fine):
        nn = s.neumann_nodes()
        pos = -np.ones(mesh.num_nodes, dtype=np.int64)
        pos[nn] = np.arange(len(nn))
        # chi = 1 on every node of an element that belongs to no other subdomain
        for e in np.nonzero(s.element_mask & ~ovl)[0]:
            loc = pos[en[e]]
            assert np.all(chis[i][loc[loc >= 0]] == 1.0), (i, e)
        A = None
        for blf in (1, 2, 3):
            _, A, B = method.fine_pencil(mesh, Ke, en, s, chis[i], blf=blf, overlap_elements=ovl)
            c = np.ones(len(nn))
            if np.linalg.norm(A @ c) <= 1e-12 * np.abs(A).max() * len(nn):
                assert c @ B @ c > 1e-8 * np.abs(A).max(), (i, blf)
                floating += blf == 1
    assert floating >= 1                        # the interior subdomains are floating


def test_single_subdomain_b2_b3_vanish():
    mesh = fem.Mesh((8, 8), 0b1)
    kap = si.channels_2d(8, 1, 1e2, seed=0)
    dec = Decomposition(mesh, (1, 1), 1, 2, (1, 1))
    chis, _ = dec.partition_of_unity()
    Ke = fem.element_matrices(mesh, kap)
    en = mesh.element_nodes()
    ovl = method.overlap_elements(dec)
    assert not ovl.any()
    assert np.all(chis[0] == 1.0)
    for blf in (2, 3):
        _, A, B = method.fine_pencil(mesh, Ke, en, dec.fine[0], chis[0], blf=blf, overlap_elements=ovl)
        assert np.abs(B).max() == 0.0
        H = method.Hierarchy(mesh, kap, (1, 1), 1, 2, (1, 1), 3, 0.3, blf=blf)
        assert H.counts(1) == [0]               # every eigenvalue is infinite


@pytest.mark.parametrize("blf,C1_of_eta", [(2, lambda eta: 1.0 + 1.0 / eta), (3, lambda eta: 2.0 * (1.0 + 1.0 / eta))])
def test_condition_bounds_b2_b3(blf, C1_of_eta):
    mesh = fem.Mesh((16, 16), 0b1)
    kap = si.channels_2d(16, 3, 1e4, seed=1)
    eta = 0.3
    H = method.Hierarchy(mesh, kap, (4, 4), 1, 2, (2, 2), 10 ** 6, eta, blf=blf)
    n = H.n
    Bm = np.stack([H.apply_preconditioner(np.eye(n)[:, j]) for j in range(n)], axis=1)
    A = H.A.toarray()
    Ls = np.linalg.cholesky(A)
    ev = np.linalg.eigvalsh(Ls.T @ (0.5 * (Bm + Bm.T)) @ Ls)
    k0, L = 4, 1
    C1 = C1_of_eta(eta)
    C = 2 * (1 + k0 * k0 * C1)
    assert ev.max() <= 1 + k0 * L + 1e-9          # Lemma upper_bound
    assert ev.min() >= 1.0 / (C ** L * (1 + k0 * C1 / (C - 1)))   # Theorem multilevelrate
