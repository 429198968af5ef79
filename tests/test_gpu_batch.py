"""Batches of independent problems on one GPU (msdd_batch_run; the multi-
problem row of the scope, with a host work queue and concurrent streams).

A reduced batch in the recipe's style (seeded sides, subdomain counts,
contrasts and log-normal + channel fields; two levels, overlap 2, nev <= 8,
eta = 0.3) is run through the batch entry point with several workers:

* every problem's result equals that of a hierarchy set up and solved on
  its own (same iterations, solutions within 1e-12 relative): running
  problems side by side changes nothing;
* on three sampled problems the CPU oracle (method mode) gives the CG
  iteration count within +-3, and the batch solution has A-norm error
  below 1e-6 against a sparse direct solve (CG stopped at 1e-8);
* statuses are per problem (maxit reached), and an invalid problem is
  rejected, by name, before any device work.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import synthetic_inputs as si
from oracle import fem, method, method_mode

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402


def small_batch(count=8, seed=11):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.choice([48, 64, 80, 96]))
        P = int(rng.integers(2, 7))
        contrast = float(10.0 ** rng.uniform(4.0, 6.0))
        w = si.Workload("small_batch_%d" % i, (N, N), (P, P), 2, 2, (1, 1), 8, 0.3,
                        seed=int(rng.integers(0, 2**31 - 1)), kind="grf", contrast=contrast,
                        extra={"n_channels": N // 16, "channel_width": 1, "n_inclusions": 0})
        out.append(w)
    return out


def _problem(w):
    return dict(n=w.n, kappa=torch.tensor(w.coefficient(), device="cuda"), parts=w.parts, overlap=w.overlap,
                levels=w.levels, group=w.group, b=pkg.assemble_rhs(w.n))


@pytest.fixture(scope="module")
def batch():
    ws = small_batch()
    probs = [_problem(w) for w in ws]
    xs, it, rel, st, sms, pms = pkg.batch_run(probs, 8, 0.3, tol=1e-8, precision=1, nworkers=4)
    return ws, probs, xs, it, rel, st


def test_batch_equals_single_problem_runs(batch):
    ws, probs, xs, it, rel, st = batch
    assert np.all(st == 0)
    for w, pr, x, k in zip(ws, probs, xs, it):
        H = pkg.Hierarchy(w.n, pr["kappa"], w.parts, w.overlap, w.levels, w.group, w.nev_max, w.eta, precision=1)
        x1, k1, _ = H.solve(pr["b"], tol=1e-8)
        H.close()
        assert k == k1, (w.name, k, k1)
        assert torch.linalg.norm(x - x1) <= 1e-12 * torch.linalg.norm(x1)


@pytest.mark.parametrize("pick", [0, 3, 6])
def test_batch_against_oracle(batch, pick):
    ws, probs, xs, it, rel, st = batch
    w = ws[pick]
    mesh = fem.Mesh(w.n, w.dirichlet_faces)
    H = method_mode.MethodModeHierarchy(mesh, w.coefficient(), w.parts, w.overlap, w.levels, w.group, w.nev_max,
                                        w.eta)
    b = fem.load_vector(mesh)
    _, it_o, *_ = method.pcg(H.A, b, H.apply_preconditioner, 1e-8)
    x = xs[pick].cpu().numpy()
    xd = spla.spsolve(H.A.tocsc(), b)
    eA = float(np.sqrt((x - xd) @ (H.A @ (x - xd)) / (xd @ (H.A @ xd))))
    print("%s: iterations %d (oracle %d), A-norm error %.2e" % (w.name, it[pick], it_o, eA))
    assert abs(int(it[pick]) - it_o) <= 3
    assert rel[pick] < 1e-8 and eA <= 1e-6


def test_batch_statuses_and_validation():
    ws = small_batch(count=3, seed=5)
    probs = [_problem(w) for w in ws]
    launches = pkg.msdd.kernel_launches()
    xs, it, rel, st, _, _ = pkg.batch_run(probs, 8, 0.3, tol=1e-8, maxit=2, nworkers=2, allow_fail=True)
    assert np.all(st == -3) and np.all(it == 2)           # MSDD_ERR_NO_CONVERGENCE per problem
    assert pkg.msdd.kernel_launches() > launches          # the workers' launches are counted
    bad = dict(probs[1])
    bad["parts"] = (1000, 1000)
    with pytest.raises(pkg.MsddError) as e:
        pkg.batch_run([probs[0], bad], 8, 0.3)
    assert e.value.status == -1 and "problem 1" in str(e.value)
