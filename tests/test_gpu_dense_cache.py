"""Dense batches (the right-looking factorisation of coarse-level matrices)
against the oracle's Cholesky solve, and the device allocation cache.

Tolerances: relative solution error 1e-10 (FP64 factors) and 1e-4 (FP32
factors) on diagonally dominant SPD matrices, as for the band solver; the
cache test checks exact equality of two identical set-ups (same kernels,
same inputs: the result must not depend on where the buffers came from).
"""
import gc

import numpy as np
import pytest

import synthetic_inputs as si
from oracle import linalg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 1e-4)])
def test_dense_batch_matches_oracle(precision, tol):
    rng = np.random.default_rng(11)
    sizes = [65, 130, 200, 257, 96]              # 3 to 9 tile rows, ragged tails
    nmax = max(sizes)
    A = np.zeros((len(sizes), nmax, nmax))
    for i, n in enumerate(sizes):
        M = rng.standard_normal((n, n))
        S = M + M.T
        S += np.diag(np.abs(S).sum(axis=1) + 1.0)
        A[i, :n, :n] = S
    B = rng.standard_normal((len(sizes), nmax, 3))
    bb = pkg.BandBatch(torch.tensor(A, device="cuda"), sizes, nmax - 1, precision=precision)
    X = torch.tensor(B, device="cuda")
    bb.solve(X)
    X = X.cpu().numpy()
    for i, n in enumerate(sizes):
        ref = linalg.cho_solve(linalg.cholesky(A[i, :n, :n]), B[i, :n])
        err = np.linalg.norm(X[i, :n] - ref.reshape(n, 3)) / np.linalg.norm(ref)
        assert err < tol, (n, err)
    bb.close()


def test_allocation_cache_reuse_and_release():
    gc.collect()                                        # batches of earlier tests release their blocks
    pkg.msdd.release_cache()
    assert pkg.msdd.cached_bytes() == 0
    w = si.channels64()
    kd = torch.tensor(w.coefficient(), device="cuda")
    b = pkg.assemble_rhs(w.n, w.dirichlet_faces)
    xs = []
    held = []
    for _ in range(2):
        H = pkg.Hierarchy(w.n, kd, w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta,
                          dirichlet_faces=w.dirichlet_faces, precision=1)
        x, it, rel = H.solve(b, tol=1e-8)
        xs.append(x.cpu().numpy())
        H.close()
        held.append(pkg.msdd.cached_bytes())
    assert held[0] > 0 and held[1] == held[0]          # the second set-up reused the first's blocks
    assert np.array_equal(xs[0], xs[1])
    pkg.msdd.release_cache()
    assert pkg.msdd.cached_bytes() == 0
