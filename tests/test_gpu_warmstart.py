"""Learned warm start of the fine subspace iteration: GPU kernels against the
oracle (oracle/warmstart.py) through the C ABI, and the gain of a network
trained by those kernels over the cold (random) start.

Tolerances: patches and start vectors 1e-6 (FP32 outputs of FP64 arithmetic);
forward 1e-5 relative (FP32 accumulation, same bfloat16 weights as the
oracle); loss 1e-5 and gradient 1e-4 relative (FP32 GEMMs over the batch);
Adam 1e-6 relative.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402
from oracle import fem  # noqa: E402
from oracle import warmstart as ws  # noqa: E402
from oracle.decomposition import Decomposition  # noqa: E402
from oracle.method import Hierarchy as OracleHierarchy  # noqa: E402
from synthetic_inputs import channels_2d, mlp_init  # noqa: E402


def boxes_of(N, parts, overlap):
    mesh = fem.Mesh((N, N), 0b1)
    dec = Decomposition(mesh, parts, overlap, 2, (1, 1))
    return mesh, dec


def test_patches_match_oracle():
    N, parts, overlap = 52, (4, 3), 2
    kappa = channels_2d(N, 6, 1e6, seed=3) * np.exp(np.random.default_rng(1).uniform(-1, 1, N * N))
    X = pkg.nn_patches((N, N), torch.tensor(kappa, device="cuda"), parts, overlap).cpu().numpy()
    _, dec = boxes_of(N, parts, overlap)
    logk = np.log10(kappa).reshape(N, N)                  # [y][x]
    for i, s in enumerate(dec.fine):
        (x0, x1), (y0, y1) = s.ext
        ref = ws.patch(logk[y0:y1, x0:x1])
        assert np.max(np.abs(X[i] - ref)) < 1e-6, i


def test_forward_loss_grad_adam_match_oracle():
    rng = np.random.default_rng(0)
    theta = mlp_init(11, ws.SHAPES)
    theta[ws.NPARAM - ws.OUT:] = (0.05 * rng.standard_normal(ws.OUT)).astype(np.float32)
    S = 37
    X = (0.3 * rng.standard_normal((S, ws.IN))).astype(np.float32)
    net = pkg.WarmStartNet(torch.tensor(theta))
    y = net.forward(torch.tensor(X)).cpu().numpy()
    y_ref, _ = ws.forward(theta.astype(np.float64), X.astype(np.float64))
    assert np.linalg.norm(y - y_ref) <= 1e-5 * np.linalg.norm(y_ref)
    m = rng.integers(0, ws.NVEC + 1, S)
    m[0], m[1] = 0, ws.NVEC
    T = np.zeros((S, ws.NVEC, ws.GRID ** 2), dtype=np.float32)
    targets = []
    for s in range(S):
        t = ws.unit_columns(rng.standard_normal((ws.GRID ** 2, m[s]))).astype(np.float32)
        T[s, :m[s]] = t.T
        targets.append(t.astype(np.float64))
    loss, grad = net.loss_grad(torch.tensor(X), torch.tensor(T), torch.tensor(m, dtype=torch.int32))
    # the oracle's mean over samples with m = 0 counts them as zero loss
    L_ref, g_ref = 0.0, np.zeros(ws.NPARAM)
    yv = ws.vectors(y_ref)
    dY = np.zeros_like(yv)
    for s in range(S):
        if m[s] == 0:
            continue
        Ls, gs = ws.sample_loss(yv[s], targets[s])
        L_ref += Ls / S
        dY[s] = gs / S
    _, cache = ws.forward(theta.astype(np.float64), X.astype(np.float64))
    g_ref = ws.backward(cache, dY.transpose(0, 2, 1).reshape(S, ws.OUT))
    assert abs(float(loss) - L_ref) <= 1e-5 * abs(L_ref)
    g = grad.cpu().numpy()
    assert np.linalg.norm(g - g_ref) <= 1e-4 * np.linalg.norm(g_ref)
    # one Adam step
    p0 = net.params.cpu().numpy().astype(np.float64)
    net.adam_step(grad, 1e-3)
    p1 = net.params.cpu().numpy()
    ref, _, _ = ws.adam(p0, g.astype(np.float64), np.zeros(ws.NPARAM), np.zeros(ws.NPARAM), 1, 1e-3)
    assert np.max(np.abs(p1 - ref)) <= 1e-6 * max(1.0, np.max(np.abs(ref)))


def test_start_vectors_match_oracle():
    N, parts, overlap = 40, (3, 2), 2
    rng = np.random.default_rng(4)
    lay = pkg.fine_layout((N, N), parts, overlap)
    Y = rng.standard_normal((lay.shape[0], ws.OUT)).astype(np.float32)
    W = pkg.nn_start_vectors((N, N), parts, overlap, torch.tensor(Y)).cpu().numpy()
    for i, (nx, ny, nz, off) in enumerate(lay):
        ref = ws.to_nodes(ws.vectors(Y[i:i + 1].astype(np.float64))[0], nx, ny)
        assert np.max(np.abs(W[off:off + nx * ny] - ref)) < 1e-6


def test_targets_span_oracle_eigenvectors():
    N, parts, overlap = 24, (3, 3), 2
    kappa = channels_2d(N, 3, 1e4, seed=2)
    H = pkg.Hierarchy((N, N), torch.tensor(kappa, device="cuda"), parts, overlap, 2, (3, 3), 6, 0.3)
    T, m = H.nn_targets()
    T, m = T.cpu().numpy(), m.cpu().numpy()
    mesh = fem.Mesh((N, N), 0b1)
    ora = OracleHierarchy(mesh, kappa, parts, overlap, 2, (3, 3), 6, 0.3)
    for i, sub in enumerate(ora.levels[ora.L].subs):
        assert m[i] == min(sub["m"], ws.NVEC)
        if m[i] == 0:
            continue
        nx = ora.dec.fine[i].neumann_box[0][1] - ora.dec.fine[i].neumann_box[0][0] + 1
        ny = ora.dec.fine[i].neumann_box[1][1] - ora.dec.fine[i].neumann_box[1][0] + 1
        Tref = ws.unit_columns(ws.to_grid(sub["W"][:, :m[i]], nx, ny))
        Tg = T[i, :m[i]].T.astype(np.float64)
        assert np.allclose(np.linalg.norm(Tg, axis=0), 1.0, atol=1e-6)
        # same span: each oracle target is reproduced by the GPU targets
        C, *_ = np.linalg.lstsq(Tg, Tref, rcond=None)
        assert np.linalg.norm(Tref - Tg @ C) < 1e-4 * np.sqrt(m[i]), i
    H.close()


def channels_problem(N, seed):
    # config-1-type field: kappa = 1 with N/8 one-element channels of kappa = 1e6
    return channels_2d(N, N // 8, 1e6, seed=seed)


def test_trained_network_reduces_subspace_iterations():
    """Trains on method-generated eigenvectors of 64 seeded channel problems
    (1024 subdomains) and compares the fine-level subspace iterations of three
    held-out problems with and without the warm start (8 FP32 start
    iterations; the warm start replaces 12 of the 16 random start columns)."""
    N, parts, overlap, nev = 128, (4, 4), 2, 12
    Xs, Ts, Ms = [], [], []
    for seed in range(64):
        kd = torch.tensor(channels_problem(N, 100 + seed), device="cuda")
        H = pkg.Hierarchy((N, N), kd, parts, overlap, 2, (4, 4), nev, 0.3, precision=1)
        T, m = H.nn_targets()
        H.close()
        Xs.append(pkg.nn_patches((N, N), kd, parts, overlap))
        Ts.append(T)
        Ms.append(m)
    X, T, M = torch.cat(Xs), torch.cat(Ts), torch.cat(Ms)
    net = pkg.WarmStartNet(torch.tensor(mlp_init(0, ws.SHAPES)))
    steps = 2000
    first = None
    for step in range(steps):
        loss, grad = net.loss_grad(X, T, M)
        net.adam_step(grad, 3e-3 * 0.5 ** (4 * step / steps))
        if step == 0:
            first = float(loss)
    assert float(net.loss_grad(X, T, M)[0]) < 0.1 * first
    counts = {"cold": 0, "warm": 0}
    for seed in (999, 998, 997):
        kd = torch.tensor(channels_problem(N, seed), device="cuda")
        H = pkg.Hierarchy((N, N), kd, parts, overlap, 2, (4, 4), nev, 0.3, precision=1)
        Th, mh = H.nn_targets()
        H.close()
        Xh = pkg.nn_patches((N, N), kd, parts, overlap)
        assert float(net.loss_grad(Xh, Th, mh)[0]) < 0.3           # held-out span error (untrained: ~0.9)
        W = pkg.nn_start_vectors((N, N), parts, overlap, net.forward(Xh))
        for name, start in (("cold", None), ("warm", W)):
            H = pkg.Hierarchy((N, N), kd, parts, overlap, 2, (4, 4), nev, 0.3, precision=1, fp32_start_iters=8,
                              warm_start=start)
            counts[name] += H.stats()["eig_iters_total"][-1]
            H.close()
    assert counts["warm"] < 0.95 * counts["cold"], counts
