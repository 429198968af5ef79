"""Degenerate cases of the method on the GPU, against the oracle.

* One subdomain covering the domain (Section 2.1 with a single fine
  subdomain): the partition of unity is 1 everywhere, so B = X Abar X = Abar
  and every eigenvalue of the local GEVP is 1.  With eta = 2 the first nev
  are selected, the preconditioner is A^{-1} plus a Galerkin coarse
  correction, BA has the eigenvalues 1 and 2 only, and CG stops after at
  most two steps, as the oracle does; the solution matches the oracle's.
* The same problem with eta = 0.3 selects nothing and the coarse space would
  be empty: set-up reports MSDD_ERR_UNSUPPORTED (the library's reading for
  empty coarse levels; the oracle runs the one-level method there).
* A zero right-hand side: x = 0 exactly, after zero CG and zero GMRES steps.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import fem, method

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402
from paper_2106_06404_gb300.msdd import MsddError  # noqa: E402


def _one_subdomain(eta):
    mesh = fem.Mesh((12, 12), 0b1)
    kap = si.channels_2d(12, 2, 1e3, seed=0)
    return mesh, kap, fem.load_vector(mesh), (mesh, kap, (1, 1), 1, 2, (1, 1), 3, eta)


def test_one_subdomain_covering_the_domain():
    mesh, kap, b, args = _one_subdomain(2.0)
    H = method.Hierarchy(*args)
    xo, ito, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-12)
    assert H.n0 == 3 and ito <= 2
    G = pkg.Hierarchy((12, 12), torch.tensor(kap, device="cuda"), (1, 1), 1, 2, (1, 1), 3, 2.0, precision=0,
                      eig_tol=1e-10)
    theta, m = G.eigenvalues(1, 0)
    assert m == 3 and np.abs(theta[:3] - 1.0).max() < 1e-10
    assert G.stats()["level_dim"][0] == 3
    x, it, rel = G.solve(torch.tensor(b, device="cuda"), tol=1e-10)
    G.close()
    print("one subdomain: GPU %d CG steps (oracle %d at 1e-12), rel. residual %.2e" % (it, ito, rel))
    assert it <= 2 and rel < 1e-10
    x = x.cpu().numpy()
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


def test_empty_coarse_space_is_reported():
    mesh, kap, b, args = _one_subdomain(0.3)
    H = method.Hierarchy(*args)
    assert H.n0 == 0                               # every eigenvalue is 1 > eta
    with pytest.raises(MsddError) as e:
        pkg.Hierarchy((12, 12), torch.tensor(kap, device="cuda"), (1, 1), 1, 2, (1, 1), 3, 0.3, precision=0)
    assert e.value.status == -7 and "empty coarse space" in str(e.value)


def test_zero_right_hand_side():
    kap = si.channels_2d(24, 3, 1e4, seed=2)
    G = pkg.Hierarchy((24, 24), torch.tensor(kap, device="cuda"), (3, 3), 2, 2, (1, 1), 6, 0.3, precision=1)
    z = torch.zeros(G.n, dtype=torch.float64, device="cuda")
    x, it, rel = G.solve(z)
    assert it == 0 and rel == 0.0 and torch.count_nonzero(x).item() == 0
    xg, itg, relg = G.solve_gmres(z)
    assert itg == 0 and relg == 0.0 and torch.count_nonzero(xg).item() == 0
    # the hierarchy still solves a nonzero system afterwards
    b = torch.tensor(fem.load_vector(fem.Mesh((24, 24), 0b1)), device="cuda")
    _, it2, rel2 = G.solve(b)
    G.close()
    assert it2 > 0 and rel2 < 1e-8
