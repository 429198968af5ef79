"""Pins of the oracle's coarse-level generating-system GEVP (Section 4.2).

On a level l < L the Neumann space of subdomain (l, i) is spanned by the
own children's coarse basis functions phi_{l+1,j,k} (j in J_{l,i}) and the
restrictions to Omega_{l,i} of the neighbouring children's ones (j in
Jbar_{l,i} minus J_{l,i}, Jbar the children whose element sets meet
T_{h,l,i}).  The oracle forms Abar_{l,i} = G^T Abar_{T_{h,l,i}} G from a
global Neumann matrix and sparse column products.  These tests rebuild the
same pencil by an independent route and check what Section 3.3 fixes:

  * the neighbour set, found by brute force over element sets;
  * Abar_{l,i} assembled element by element over T_{h,l,i}, each
    neighbour function explicitly restricted (zeroed outside the closure of
    Omega_{l,i}) and each own function taken whole;
  * B_{l,i} = X Abar_{l,i} X with X the own-generator mask;
  * the own-own block of Abar_{l,i} equals the coarse Dirichlet matrix
    A_{l,i} (own functions vanish outside Omega_{l,i}), which the oracle
    takes from the Galerkin matrix instead;
  * the spectrum structure of the pencil with ker A cap ker B != {0}: on
    the complement of the common kernel, #finite eigenvalues = rank B and
    #(lambda = 0) = rank(A + B) - rank A (the non-defectiveness lemma and
    the spectrum display after it, with ranks from numpy's SVD);
  * brute force: scipy's LAPACK symmetric-definite solver on the
    rank-reduced, spectrally transformed pencil;
  * the projection stability estimates (Lemma gevp_properties) for the
    oracle's eigenvectors on random vectors;
  * the regularised LDL^T route of Section 4.2 (Eq. evp_reg) that the
    oracle takes on coarse levels: on generators with exact dependencies it
    drops exactly those (null pivots = dim ker A cap ker B) and yields the
    pencil's eigenvalues on the span, whatever the generators' scaling;
  * in 3D the threshold (a pivot d_k <= 1e-6 K_kk is null) also drops
    generators that are only nearly dependent; there the null pivots are
    recomputed as explicit Schur complements of K = Abar + sigma B onto the
    generators kept before them, and the finite eigenvalues as those of the
    Schur complement of Abar onto the own generators (B vanishes outside
    that block) against B's own block, by scipy's symmetric-definite
    solver; a pencil restricted to fewer generators has eigenvalues no
    lower, one by one, than the pencil with every generator kept (the
    Courant-Fischer characterisation), which the hierarchy built with a
    threshold that keeps them all must show.  The 2D spectrum-structure and
    brute-force pins assume exact dependencies only and stay on the 2D
    cases.
"""
import numpy as np
import pytest
import scipy.linalg as sla

import synthetic_inputs as si
from oracle import fem, method


@pytest.fixture(scope="module")
def three_level():
    mesh = fem.Mesh((16, 16), 0b1)
    kap = si.channels_2d(16, 3, 1e4, seed=1)
    H = method.Hierarchy(mesh, kap, (4, 4), 1, 3, (2, 2), 6, 0.3, keep_local=True)
    return mesh, kap, H


@pytest.fixture(scope="module")
def ragged_three_level():
    # 2 x 2 middle subdomains with 3 and 2 children along x (uneven groups)
    mesh = fem.Mesh((20, 18), 0b1)
    kap = si.channels_2d(20, 3, 1e5, seed=4)[: 20 * 18]
    H = method.Hierarchy(mesh, kap, (5, 4), 2, 3, (2, 2), 5, 0.3, keep_local=True)
    return mesh, kap, H


@pytest.fixture(scope="module")
def three_level_3d():
    # 8^3 elements, 4^3 fine subdomains, 2^3 middle subdomains of 2^3 children
    mesh = fem.Mesh((8, 8, 8), 0b1)
    kap = si.layered_3d(8, seed=2)
    H = method.Hierarchy(mesh, kap, (4, 4, 4), 1, 3, (2, 2, 2), 4, 0.3, keep_local=True)
    return mesh, kap, H


def _node_functions(mesh, H, l):
    """Level-(l+1) coarse basis functions phi_{l+1,j,k} as nodal arrays over all
    mesh nodes (zero on Dirichlet nodes), one list per child j."""
    P = H.levels[l + 1].P_coarse.toarray()       # unknown coordinates
    n2u = H.n2u
    out = []
    for a, b in H.levels[l + 1].col_range:
        cols = []
        for c in range(a, b):
            v = np.zeros(mesh.num_nodes)
            on = n2u >= 0
            v[on] = P[n2u[on], c]
            cols.append(v)
        out.append(cols)
    return out


def _child_masks(H, l):
    return H.dec.element_mask[l + 1]


def _independent_pencil(mesh, kap, H, l, i):
    """(own children, neighbour children, Abar, B) of subdomain (l, i) from an
    element loop over T_{h,l,i}."""
    dec = H.dec
    mask = dec.element_mask[l][i]
    own = list(dec.members[l][i])
    kids = _child_masks(H, l)
    nbr = sorted(j for j in range(len(kids)) if j not in own and np.any(kids[j] & mask))
    en = mesh.element_nodes()
    # closure of Omega_{l,i}: nodes of its elements
    closure = np.zeros(mesh.num_nodes, dtype=bool)
    closure[np.unique(en[mask])] = True
    phis = _node_functions(mesh, H, l)
    gens = [phi for j in own for phi in phis[j]]
    n_own = len(gens)
    gens += [np.where(closure, phi, 0.0) for j in nbr for phi in phis[j]]
    G = np.stack(gens, axis=1) if gens else np.zeros((mesh.num_nodes, 0))
    Ke = fem.element_matrices(mesh, kap)
    Abar = np.zeros((G.shape[1], G.shape[1]))
    for e in np.nonzero(mask)[0]:
        Ge = G[en[e]]                              # element nodal values of every generator
        Abar += Ge.T @ Ke[e] @ Ge
    x = np.zeros(G.shape[1])
    x[:n_own] = 1.0
    B = x[:, None] * Abar * x[None, :]
    return own, nbr, Abar, B, n_own


def _cases(H):
    return range(H.dec.num_subdomains(1))


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level", "three_level_3d"])
def test_generating_system_matches_element_assembly(fixture, request):
    mesh, kap, H = request.getfixturevalue(fixture)
    lev = H.levels[1]
    for i in _cases(H):
        own, nbr, Abar, B, n_own = _independent_pencil(mesh, kap, H, 1, i)
        s = lev.subs[i]
        assert list(s["own"]) == own
        assert list(s["nbr"]) == nbr
        scale = max(1.0, np.abs(Abar).max())
        assert s["Abar"].shape == Abar.shape
        assert np.abs(s["Abar"] - Abar).max() <= 1e-11 * scale, i
        assert np.abs(s["B"] - B).max() <= 1e-11 * scale, i
        # own functions vanish outside Omega_{l,i}: Neumann own block = Dirichlet matrix
        assert np.abs(s["Ai"] - Abar[:n_own, :n_own]).max() <= 1e-10 * scale, i


def _rank(M, rel=1e-9):
    s = np.linalg.svd(M, compute_uv=False)
    if s.size == 0 or s[0] == 0.0:
        return 0, s
    return int(np.sum(s > rel * s[0])), s


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level"])
def test_coarse_spectrum_structure(fixture, request):
    """Spectrum of the generating-system pencil on the complement of
    ker A cap ker B: rank B finite eigenvalues, rank(A+B) - rank A zeros."""
    mesh, kap, H = request.getfixturevalue(fixture)
    checked_zero = False
    for s in H.levels[1].subs:
        A, B = s["Abar"], s["B"]
        rAB, sAB = _rank(A + B)
        rA, sA = _rank(A)
        rB, sB = _rank(B)
        # the ranks are numerically unambiguous on these cases
        for r, sv in ((rAB, sAB), (rA, sA), (rB, sB)):
            if r < len(sv):
                assert sv[r] < 1e-11 * sv[0] and sv[r - 1] > 1e-7 * sv[0]
        lam = s["lam"]
        assert len(lam) == rB
        zeros = int(np.sum(lam < 1e-8))
        assert zeros == rAB - rA
        checked_zero = checked_zero or zeros > 0
        assert np.all(lam >= -1e-9)
    assert checked_zero                           # some floating middle subdomain


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level"])
def test_coarse_eigenvalues_brute_force(fixture, request):
    mesh, kap, H = request.getfixturevalue(fixture)
    for s in H.levels[1].subs:
        A, B = s["Abar"], s["B"]
        S = A + B
        w, U = np.linalg.eigh(S)
        U = U[:, w > 1e-9 * w.max()]
        mu = sla.eigh(U.T @ B @ U, U.T @ S @ U, eigvals_only=True)
        mu = np.sort(mu[mu > 1e-10])[::-1]
        lam_ref = 1.0 / mu - 1.0
        lam = s["lam"]
        assert len(lam) == len(lam_ref)
        k = min(len(lam), 12)
        err = np.abs(lam[:k] - lam_ref[:k]) / np.maximum(np.abs(lam_ref[:k]), 1e-6)
        assert err.max() < 1e-7, err


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level", "three_level_3d"])
def test_coarse_projection_stability(fixture, request):
    """|Pi_m v|_a <= |v|_a, |v - Pi_m v|_a <= |v|_a and, for m >= #zeros,
    |v - Pi_m v|_b^2 <= |v - Pi_m v|_a^2 / lambda_{m+1} (Lemma gevp_properties)."""
    mesh, kap, H = request.getfixturevalue(fixture)
    rng = np.random.default_rng(0)
    for s in H.levels[1].subs:
        A, B = s["Abar"], s["B"]
        # full eigenvector set of the finite part, b-orthonormal
        lam, W = method.gevp(A, B, rank_reveal=True)
        assert np.allclose(W.T @ B @ W, np.eye(len(lam)), atol=1e-7)
        r = int(np.sum(lam < 1e-8))
        an = lambda v: np.sqrt(max(v @ A @ v, 0.0))
        bn2 = lambda v: max(v @ B @ v, 0.0)
        for _ in range(5):
            v = rng.standard_normal(A.shape[0])
            for m in range(0, len(lam)):
                Pv = W[:, :m] @ (W[:, :m].T @ (B @ v))
                assert an(Pv) <= an(v) * (1 + 1e-8) + 1e-12
                assert an(v - Pv) <= an(v) * (1 + 1e-8) + 1e-12
                if m >= r and m < len(lam):
                    d = v - Pv
                    assert bn2(d) <= an(d) ** 2 / lam[m] * (1 + 1e-7) + 1e-12


def _dependent_pencil(rng, scales=None):
    """A = G^T Sa G, B = G^T Sb G on generators G (columns) with exact
    dependencies: ker A cap ker B = ker G."""
    m, k = 30, 12
    G = rng.standard_normal((m, k))
    G = np.concatenate([G, G[:, [0]] + G[:, [1]], 3.0 * G[:, [4]], G[:, [2]] - 0.5 * G[:, [7]]], axis=1)
    M = rng.standard_normal((m, m))
    Sa = M @ M.T + m * np.eye(m)
    mask = np.zeros(m)
    mask[: m // 2] = 1.0
    Sb = mask[:, None] * Sa * mask[None, :]
    A, B = G.T @ Sa @ G, G.T @ Sb @ G
    if scales is not None:
        A = scales[:, None] * A * scales[None, :]
        B = scales[:, None] * B * scales[None, :]
        G = G * scales[None, :]
    return G, Sa, Sb, A, B


def test_regularised_gevp_equals_pencil_on_the_span():
    """Section 4.2: with dependent generators the regularised LDL^T drops
    exactly the dependencies (3 null pivots here), and the eigenvalues are
    those of the pencil on span(G) (orthonormal basis by SVD, scipy's
    symmetric-definite solver); a rescaling of the generators changes
    nothing."""
    rng = np.random.default_rng(3)
    G, Sa, Sb, A, B = _dependent_pencil(rng)
    U, s, _ = np.linalg.svd(G, full_matrices=False)
    Q = U[:, s > 1e-10 * s[0]]
    ref = sla.eigh(Q.T @ Sa @ Q, Q.T @ (Sa + Sb) @ Q, eigvals_only=True)   # mu-type: a = nu (a + b)
    nu = np.sort(ref)
    mu_b = 1.0 - nu                                # b = (1 - nu)(a + b)
    fin = mu_b > 1e-12
    lam_ref = np.sort(nu[fin] / mu_b[fin])
    lam, W, nnull = method.gevp_regularised(A, B, 1e-2, 1e-10)
    assert nnull == G.shape[1] - Q.shape[1] == 3
    assert len(lam) == len(lam_ref)
    assert np.allclose(lam, lam_ref, rtol=1e-8, atol=1e-10)
    assert np.allclose(W.T @ B @ W, np.eye(len(lam)), atol=1e-8)
    assert np.allclose(A @ W, (B @ W) * lam[None, :], atol=1e-7 * np.abs(A).max())
    scales = np.exp(rng.uniform(np.log(1e-6), np.log(1e3), G.shape[1]))
    _, _, _, As, Bs = _dependent_pencil(np.random.default_rng(3), scales)
    lam_s, _, nnull_s = method.gevp_regularised(As, Bs, 1e-2, 1e-10)
    assert nnull_s == 3 and np.allclose(lam_s, lam, rtol=1e-7, atol=1e-10)


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level"])
def test_null_pivots_are_the_common_kernel(fixture, request):
    """On these cases every null pivot is an exact dependency: their number
    is dim(ker A cap ker B) = n - rank(A + B)."""
    mesh, kap, H = request.getfixturevalue(fixture)
    for s in H.levels[1].subs:
        A, B = s["Abar"], s["B"]
        rAB, _ = _rank(A + B)
        assert s["null_pivots"] == A.shape[0] - rAB


def _schur_route(A, B, sigma, tau):
    """(number of null pivots, finite eigenvalues ascending) of the pencil
    (A, B) by explicit Schur complements: generator k is null when
    K_kk - K_kS K_SS^{-1} K_Sk <= tau K_kk, S the generators kept before it;
    the finite eigenvalues are those of A_oo - A_on A_nn^{-1} A_no against
    B_oo on the kept own (o) and neighbour (n) generators."""
    n = A.shape[0]
    no = int(np.sum(np.diag(B) > 0))
    assert np.all(B[no:, :] == 0.0) and np.all(B[:, no:] == 0.0)     # B lives on the own block
    K = A + sigma * B
    kept = []
    for k in range(n):
        d = K[k, k]
        if kept:
            d -= K[k, kept] @ np.linalg.solve(K[np.ix_(kept, kept)], K[kept, k])
        if d > tau * K[k, k]:
            kept.append(k)
    ko = [k for k in kept if k < no]
    kn = [k for k in kept if k >= no]
    S = A[np.ix_(ko, ko)]
    if kn:
        Aon = A[np.ix_(ko, kn)]
        S = S - Aon @ np.linalg.solve(A[np.ix_(kn, kn)], Aon.T)
    lam = sla.eigh(0.5 * (S + S.T), B[np.ix_(ko, ko)], eigvals_only=True)
    return n - len(kept), np.sort(lam)


@pytest.mark.parametrize("fixture", ["three_level", "ragged_three_level", "three_level_3d"])
def test_coarse_eigenvalues_schur_complement(fixture, request):
    mesh, kap, H = request.getfixturevalue(fixture)
    for i, s in enumerate(H.levels[1].subs):
        nnull, lam_ref = _schur_route(s["Abar"], s["B"], H.sigma, H.reg_tol)
        assert s["null_pivots"] == nnull, i
        lam = s["lam"]
        assert len(lam) == len(lam_ref), i
        err = np.abs(lam - lam_ref) / np.maximum(np.abs(lam_ref), 1e-6)
        assert err.max() < 1e-8, (i, err)


def test_three_d_threshold_drops_near_dependencies(three_level_3d):
    mesh, kap, H = three_level_3d
    assert H.reg_tol == 1e-6
    near = 0
    for s in H.levels[1].subs:
        rAB, _ = _rank(s["Abar"] + s["B"])
        near += s["null_pivots"] - (s["Abar"].shape[0] - rAB)
    assert near > 0                              # null pivots that are not exact dependencies
    full = method.Hierarchy(mesh, kap, (4, 4, 4), 1, 3, (2, 2, 2), 4, 0.3, reg_tol=1e-10, keep_local=True)
    for s, f in zip(H.levels[1].subs, full.levels[1].subs):
        assert f["null_pivots"] == 0 and np.array_equal(s["Abar"], f["Abar"])
        lo, hi = f["lam"], s["lam"]
        assert len(hi) == len(lo)               # rank B: the own generators are all kept
        assert np.all(hi >= lo - 1e-9 * np.maximum(1.0, np.abs(lo)))
