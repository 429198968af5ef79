"""Pins of the warm-start oracle (oracle/warmstart.py) against definitions
that do not go through its own code: bfloat16 rounding of exact binary
values, area averaging of linear fields, finite differences, the subspace
invariance of the loss, exactness of bilinear interpolation on bilinear
fields and the closed form of a first Adam step."""
import numpy as np
import pytest

from oracle import warmstart as ws
from synthetic_inputs import mlp_init


def test_bf16_round_exact_values():
    e = 2.0 ** -8                                       # half a bf16 ulp at 1
    x = np.array([1.0, 1 + e, 1 + 3 * e, 1 + 2 * e, -1 - 3 * e, 3.0, 1e-3, 0.0], dtype=np.float32)
    r = ws.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                                  # tie -> even mantissa
    assert r[2] == 1 + 4 * e                            # tie -> even (up)
    assert r[3] == 1 + 2 * e                            # representable
    assert r[4] == -(1 + 4 * e)
    assert r[5] == 3.0 and r[7] == 0.0
    rng = np.random.default_rng(0)
    y = rng.standard_normal(10000).astype(np.float32)
    ry = ws.bf16_round(y)
    assert np.all(np.abs(ry - y) <= 2.0 ** -8 * np.abs(y) * (1 + 1e-7))      # unit roundoff of 8-bit significands
    assert np.array_equal(ws.bf16_round(ry.astype(np.float32)), ry)


def test_patch_area_average_by_supersampling():
    # each element split into PATCH x PATCH equal sub-cells: every patch cell
    # is then exactly ny x nx sub-cells, so its average is a plain mean
    rng = np.random.default_rng(5)
    for ny, nx in ((36, 36), (20, 20), (30, 17)):
        f = rng.standard_normal((ny, nx))
        fine = np.repeat(np.repeat(f, ws.PATCH, 0), ws.PATCH, 1)
        ref = fine.reshape(ws.PATCH, ny, ws.PATCH, nx).mean(axis=(1, 3))
        p = ws.patch(f).reshape(ws.PATCH, ws.PATCH) * 6.0
        assert np.allclose(p, ref - ref.mean(), atol=1e-12)
    assert np.allclose(ws.patch(np.full((36, 36), 5.0)), 0.0)


def test_sample_loss_invariance_and_limits():
    rng = np.random.default_rng(1)
    Y = rng.standard_normal((ws.GRID ** 2, ws.NVEC))
    T = ws.unit_columns(rng.standard_normal((ws.GRID ** 2, 5)))
    L, _ = ws.sample_loss(Y, T)
    Q = rng.standard_normal((ws.NVEC, ws.NVEC)) + 3 * np.eye(ws.NVEC)
    L2, _ = ws.sample_loss(Y @ Q, T)
    assert abs(L - L2) < 1e-6
    Tin = ws.unit_columns(Y @ rng.standard_normal((ws.NVEC, 4)))
    assert ws.sample_loss(Y, Tin)[0] < 1e-6
    # targets orthogonal to span(Y): the loss is 1 per unit column
    Qy, _ = np.linalg.qr(Y, mode="complete")
    Tout = Qy[:, ws.NVEC:ws.NVEC + 3]
    assert abs(ws.sample_loss(Y, Tout)[0] - 1.0) < 1e-9


def test_sample_loss_gradient_finite_differences():
    rng = np.random.default_rng(2)
    Y = rng.standard_normal((ws.GRID ** 2, ws.NVEC))
    T = ws.unit_columns(rng.standard_normal((ws.GRID ** 2, 6)))
    _, g = ws.sample_loss(Y, T)
    h = 1e-6
    for _ in range(20):
        i, j = rng.integers(Y.shape[0]), rng.integers(Y.shape[1])
        Yp, Ym = Y.copy(), Y.copy()
        Yp[i, j] += h
        Ym[i, j] -= h
        fd = (ws.sample_loss(Yp, T)[0] - ws.sample_loss(Ym, T)[0]) / (2 * h)
        assert abs(fd - g[i, j]) <= 1e-6 * max(1.0, abs(fd))


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(3)
    theta = mlp_init(4, ws.SHAPES).astype(np.float64)
    theta[ws.NPARAM - ws.OUT:] = 0.1 * rng.standard_normal(ws.OUT)   # non-zero output bias
    X = 0.3 * rng.standard_normal((3, ws.IN))
    targets = [ws.unit_columns(rng.standard_normal((ws.GRID ** 2, k))) for k in (3, 5, 8)]
    L, g = ws.loss_and_grad(theta, X, targets, round_weights=False)
    h = 1e-6
    idx = np.concatenate([rng.integers(0, ws.NPARAM, 40), np.arange(ws.NPARAM - 5, ws.NPARAM)])
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (ws.loss_and_grad(tp, X, targets, False)[0] - ws.loss_and_grad(tm, X, targets, False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 2e-6 * max(1e-3, abs(fd)) + 1e-9, (i, fd, g[i])


def test_bilinear_exact_on_bilinear_fields():
    g = np.arange(ws.GRID) / (ws.GRID - 1)
    gy, gx = np.meshgrid(g, g, indexing="ij")
    f = lambda u, v: 1.5 - 2 * u + 0.5 * v + 3 * u * v
    G = f(gx, gy).reshape(-1, 1)
    for nx, ny in ((37, 37), (21, 19)):
        vals = ws.to_nodes(G, nx, ny)[:, 0]
        u = np.tile(np.arange(nx) / (nx - 1), ny)
        v = np.repeat(np.arange(ny) / (ny - 1), nx)
        assert np.allclose(vals, f(u, v), atol=1e-13)
        back = ws.to_grid(f(u, v).reshape(-1, 1), nx, ny)
        assert np.allclose(back[:, 0], G[:, 0], atol=1e-13)


def test_adam_first_step_closed_form():
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    t1, m, v = ws.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01)
    # bias-corrected first step: m_hat = g, v_hat = g^2
    assert np.allclose(t1, theta - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
