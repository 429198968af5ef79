"""Parity at the full size of the 2D benchmark workload, in the configuration
bench.py times: grf2d 512 x 512 elements (262,656 unknowns), 16 x 16 fine
subdomains, overlap 2, 3 levels (4 x 4 groups), nev <= 12, eta = 0.3, chosen
form (FP32 local factors, FP64 outer iteration).

The oracle cannot run the whole set-up at this size (256 dense GEVPs of
order ~1369 by Jacobi), so these tests check what it can compute one item
at a time, on sampled fine subdomains, plus properties that hold at any
size:

* Ritz values: by Sylvester's law of inertia (Section 3.3: the pencil
  (Abar_i, B_i) has ker Abar_i and ker B_i meeting only in 0 on the fine
  level), the number of negative eigenvalues of Abar_i - t B_i is the number
  of pencil eigenvalues below t.  Every selected GPU Ritz value theta_k must
  satisfy  #{lambda < theta_k - d_k} <= k - 1  and  #{lambda < theta_k + d_k} >= k,
  which fails for a wrong or missed eigenvalue (d_k = 1e-6 (theta_k + sigma),
  the stated eigenvalue tolerance; the error of a Ritz value is of second
  order in its residual, which is below 1e-6).
* Selection count (Eq. coarse_space_def): m_i = min(nev_max, #{lambda < eta})
  exactly, from the inertia at eta (+-1 only if an eigenvalue lies within
  1e-6 eta of eta).
* Normalisation b(w, w) = 1 (Section 3.3): the exported coarse basis functions
  phi_k = chi w_k satisfy phi^T Abar_i phi = I.
* The global operator applied by the library equals the oracle's assembled
  matrix, and the PCG solution of the oracle's load vector meets the stopping
  rule (Section 5: the CG residual below 1e-8 ||b||).  The true residual of
  any FP64 CG iterate is limited by rounding to about
  eps ||(|A| |x|)|| / ||b|| (the residual gap of the recursively updated
  residual; ~7e-7 here because the coefficient contrast is 1e6), so it is
  checked against that bound, evaluated in extended precision, and the
  Jacobi-scaled true residual against 1e-8.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402
from oracle import fem, linalg  # noqa: E402
from oracle.decomposition import Decomposition  # noqa: E402
from oracle.method import fine_pencil  # noqa: E402
from synthetic_inputs import grf512  # noqa: E402

SIGMA = 1e-2
SAMPLE = (0, 15, 120, 137, 255)


@pytest.fixture(scope="module")
def case():
    w = grf512()
    kappa = w.coefficient()
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    H = pkg.Hierarchy(w.n, torch.tensor(kappa, device="cuda"), w.parts, w.overlap, w.levels, w.group,
                      w.nev_max, w.eta, dirichlet_faces=w.dirichlet_faces, precision=1, sigma=SIGMA)
    dec = Decomposition(mesh, w.parts, w.overlap, w.levels, w.group)
    chis, _ = dec.partition_of_unity()
    Ke = fem.element_matrices(mesh, kappa)
    en = mesh.element_nodes()
    pencils = {i: fine_pencil(mesh, Ke, en, dec.fine[i], chis[i]) for i in SAMPLE}
    yield w, kappa, mesh, H, pencils
    H.close()


def count_below(Abar, B, t):
    return linalg.negative_count(Abar - t * B)


@pytest.mark.parametrize("i", SAMPLE)
def test_fine_ritz_values_bracketed_by_inertia(case, i):
    w, _, _, H, pencils = case
    _, Abar, B = pencils[i]
    L = w.levels - 1
    theta, m = H.eigenvalues(L, i)
    assert m >= 1
    for k in range(1, m + 1):
        th = theta[k - 1]
        d = 1e-6 * (th + SIGMA)
        assert count_below(Abar, B, th - d) <= k - 1, (i, k, th)
        assert count_below(Abar, B, th + d) >= k, (i, k, th)


@pytest.mark.parametrize("i", SAMPLE)
def test_fine_selection_count_exact(case, i):
    w, _, _, H, pencils = case
    _, Abar, B = pencils[i]
    _, m = H.eigenvalues(w.levels - 1, i)
    lo = min(w.nev_max, count_below(Abar, B, w.eta * (1 - 1e-6)))
    hi = min(w.nev_max, count_below(Abar, B, w.eta * (1 + 1e-6)))
    assert lo <= m <= hi, (i, m, lo, hi)
    if lo == hi:
        assert m == min(w.nev_max, count_below(Abar, B, w.eta))


@pytest.mark.parametrize("i", SAMPLE)
def test_fine_basis_b_orthonormal(case, i):
    _, _, mesh, H, pencils = case
    nn, Abar, _ = pencils[i]
    phi = H.fine_basis(i)
    u = mesh.node_to_unknown()[nn]
    assert np.all(u >= 0)
    P = phi[u]                                  # chi w on the subdomain's Neumann nodes
    G = P.T @ Abar @ P                          # b(w_j, w_k) = abar(chi w_j, chi w_k)
    assert np.max(np.abs(G - np.eye(G.shape[0]))) < 1e-8
    # nothing outside the subdomain
    outside = np.ones(phi.shape[0], dtype=bool)
    outside[u] = False
    assert np.all(phi[outside] == 0.0)


def test_operator_and_pcg_solution(case):
    w, kappa, mesh, H, _ = case
    A = fem.assemble_system(mesh, kappa)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(A.shape[0])
    y = H.apply_operator(torch.tensor(x, device="cuda")).cpu().numpy()
    ref = A @ x
    assert np.linalg.norm(y - ref) <= 1e-13 * np.linalg.norm(ref)
    b = fem.load_vector(mesh)
    xs, it, rel = H.solve(torch.tensor(b, device="cuda"), tol=1e-8)
    xs = xs.cpu().numpy()
    assert rel < 1e-8
    assert 10 <= it <= 200
    # true residual in extended precision (no rounding of its own at this level)
    ax = np.add.reduceat(A.data.astype(np.longdouble) * xs[A.indices].astype(np.longdouble), A.indptr[:-1])
    res = b.astype(np.longdouble) - ax
    true_rel = float(np.sqrt(np.sum(res * res)) / np.linalg.norm(b))
    gamma = np.linalg.norm(abs(A) @ np.abs(xs)) / np.linalg.norm(b)
    assert true_rel <= 1e-8 + 10 * np.finfo(np.float64).eps * gamma, (true_rel, gamma)
    d = np.sqrt(A.diagonal())
    scaled = float(np.sqrt(np.sum((res / d) ** 2))) / np.linalg.norm(b / d)
    assert scaled < 1e-8, scaled
    st = H.stats()
    assert st["level_dim"][-1] == A.shape[0]
    assert st["eig_unconverged"] == [0] * w.levels
