"""Full-size parity of the 512 x 512 workload (262,656 unknowns, 16 x 16
fine subdomains, three levels) against the oracle's method mode, which runs
the whole set-up on the host cores (band Cholesky and block subspace
iteration on the fine level, the exact regularised generating-system GEVPs
of Section 4.2 on the middle level, Galerkin and coarsest factors, CG).

* Plain FP64 form with a tight eigen-residual tolerance (1e-9): every
  selected eigenvalue of all 256 fine subdomains to 1e-6 relative (floor
  1e-3 eta), every count and coarse dimension exact, CG iterations within
  +-3, the solution's A-norm error against a sparse direct solve below
  1e-6.  Middle-level eigenvalues to 1e-4: their pencils are built from the
  fine coarse spaces, whose spans both sides know only to the fine
  eigen-residuals over the spectral gaps at eta (the residuals of this
  workload, contrast ~1e10, stop near 1e-10 on either side, and the
  oracle's at 1e-8), so they agree to ~2.5e-5 (measured), not to 1e-6.
* Chosen form (bench defaults, eigen-residual 1e-6): fine eigenvalues to
  1e-6 and all counts and dimensions exact.  Its middle-level eigenvalues
  come from generating systems built from fine eigenvectors that are only
  accurate to the residual over the spectral gaps, so they are reported,
  not held to a bound here (2.8e-4 measured).
"""
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402
from oracle import fem, method, method_mode  # noqa: E402
from synthetic_inputs import grf512  # noqa: E402


@pytest.fixture(scope="module")
def oracle():
    w = grf512()
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    kap = w.coefficient()
    H = method_mode.MethodModeHierarchy(mesh, kap, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                                        processes=os.cpu_count() or 1)
    b = fem.load_vector(mesh)
    _, it, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-8)
    xd = spla.spsolve(H.A.tocsc(), b)
    return w, kap, H, b, it, xd


def _compare(G, H, w, lev):
    worst, mism = 0.0, []
    for i, s in enumerate(H.levels[lev].subs):
        theta, m = G.eigenvalues(lev, i)
        if m != s["m"]:
            mism.append((i, m, s["m"]))
            continue
        if m:
            lam = s["lam"][:m]
            worst = max(worst, float(np.max(np.abs(theta[:m] - lam) / np.maximum(np.abs(lam), 1e-3 * w.eta))))
    return worst, mism


@pytest.mark.parametrize("precision,eig_tol", [(0, 1e-9), (1, 1e-6)])
def test_fullsize_against_method_mode_oracle(oracle, precision, eig_tol):
    w, kap, H, b, it_o, xd = oracle
    G = pkg.Hierarchy(w.n, torch.tensor(kap, device="cuda"), w.parts, w.overlap, w.levels, w.group, w.nev_max,
                      w.eta, dirichlet_faces=w.dirichlet_faces, precision=precision, eig_tol=eig_tol)
    st = G.stats()
    fine_err, fine_mism = _compare(G, H, w, w.levels - 1)
    mid_err, mid_mism = _compare(G, H, w, 1)
    x, it, rel = G.solve(torch.tensor(b, device="cuda"), tol=1e-8)
    x = x.cpu().numpy()
    eA = float(np.sqrt((x - xd) @ (H.A @ (x - xd)) / (xd @ (H.A @ xd))))
    print("precision %d eig_tol %.0e: fine eig err %.2e, middle eig err %.2e, mismatches %s %s, dims %s vs %s, "
          "iterations %d vs %d, A-norm error %.2e" % (precision, eig_tol, fine_err, mid_err, fine_mism, mid_mism,
                                                      st["level_dim"], [H.coarse_dims()[0], H.coarse_dims()[1]],
                                                      it, it_o, eA))
    assert fine_mism == [] and mid_mism == []
    assert st["level_dim"][0] == H.coarse_dims()[0] and st["level_dim"][1] == H.coarse_dims()[1]
    assert fine_err <= 1e-6
    if precision == 0:
        assert mid_err <= 1e-4
        assert abs(it - it_o) <= 3
    assert rel < 1e-8 and eA <= 1e-6
    G.close()
