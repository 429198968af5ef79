"""Learned warm start of the fine-level subspace iteration (oracle).

TEST INFRASTRUCTURE ONLY: imported by tests/, never by the product path.

The paper has no learned component; this is the follow-on direction that
starts the batched subspace iteration for the fine GEVPs (Eq. theGEVP) from
predicted vectors instead of random ones.  Every piece is written in FP64 from
its definition:

* patch: the subdomain's log10 kappa on its element box, area-averaged onto a
  PATCH x PATCH grid of equal cells (exact overlap areas), minus its mean,
  divided by 6 (the decades of the contrast range);
* network: MLP  PATCH^2 -> HIDDEN -> HIDDEN -> NVEC * GRID^2  with ReLU,
  weights rounded to bfloat16 (round to nearest even) before use, biases and
  arithmetic in full precision;
* output: NVEC vectors on a GRID x GRID node grid over the subdomain's
  Neumann box (unit square), bilinearly interpolated to its nodes;
* loss of one sample (subspace-invariant, sign and rotation free): with the
  predicted Y (GRID^2 x NVEC) and the unit-norm targets T (GRID^2 x m),
      L = min_C ||T - Y C||_F^2 + eps ||C||_F^2,   C = (Y^T Y + eps I)^{-1} Y^T T,
  divided by m; by the envelope theorem dL/dY = -2 (T - Y C) C^T / m;
  the batch loss is the mean over samples;
* Adam (Kingma & Ba) with bias correction.
"""
import numpy as np

PATCH, HIDDEN, GRID, NVEC = 24, 48, 13, 12
IN, OUT = PATCH * PATCH, NVEC * GRID * GRID
SHAPES = [(HIDDEN, IN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (OUT, HIDDEN), (OUT,)]
NPARAM = int(sum(np.prod(s) for s in SHAPES))
EPS_LS = 1e-6


def unpack(theta):
    """Flat parameter vector -> [W1, b1, W2, b2, W3, b3] (views, row-major)."""
    out, o = [], 0
    for s in SHAPES:
        n = int(np.prod(s))
        out.append(theta[o:o + n].reshape(s))
        o += n
    return out


def bf16_round(x):
    """Round float32 values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    bias = 0x7FFF + ((u >> 16) & 1)
    r = ((u + bias) & 0xFFFF0000).astype(np.uint32)
    finite = np.isfinite(np.asarray(x, dtype=np.float32))
    r = np.where(finite, r, np.asarray(x, dtype=np.float32).view(np.uint32))
    return r.view(np.float32).astype(np.float64)


def _overlap_weights(w, n):
    """(n, w) averaging weights: row I = overlap of cell [I w/n, (I+1) w/n) with
    element [e, e+1), divided by the cell length."""
    W = np.zeros((n, w))
    for I in range(n):
        a, b = I * w / n, (I + 1) * w / n
        for e in range(int(np.floor(a)), min(w, int(np.ceil(b)))):
            W[I, e] = max(0.0, min(b, e + 1) - max(a, e))
        W[I] /= (b - a)
    return W


def patch(logk_box):
    """Network input of one subdomain: logk_box is (ny, nx) log10 kappa of its
    element box (x fastest along the second axis)."""
    ny, nx = logk_box.shape
    P = _overlap_weights(ny, PATCH) @ logk_box @ _overlap_weights(nx, PATCH).T
    return ((P - P.mean()) / 6.0).ravel()


def forward(theta, X, round_weights=True):
    """Batch forward; X (S, IN).  Returns outputs (S, OUT) and the cache."""
    W1, b1, W2, b2, W3, b3 = unpack(theta)
    if round_weights:
        W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    a1 = X @ W1.T + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2.T + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3.T + b3
    return y, (X, a1, h1, a2, h2, W1, W2, W3)


def backward(cache, dy):
    """Gradient of the parameters (flat, straight through the bf16 rounding)."""
    X, a1, h1, a2, h2, W1, W2, W3 = cache
    dW3 = dy.T @ h2
    db3 = dy.sum(0)
    da2 = (dy @ W3) * (a2 > 0)
    dW2 = da2.T @ h1
    db2 = da2.sum(0)
    da1 = (da2 @ W2) * (a1 > 0)
    dW1 = da1.T @ X
    db1 = da1.sum(0)
    return np.concatenate([g.ravel() for g in (dW1, db1, dW2, db2, dW3, db3)])


def vectors(y):
    """(S, OUT) outputs -> (S, GRID^2, NVEC) grid vectors (vector k at k * GRID^2)."""
    return y.reshape(-1, NVEC, GRID * GRID).transpose(0, 2, 1)


def sample_loss(Y, T):
    """Loss and dL/dY of one sample (Y: GRID^2 x NVEC, T: GRID^2 x m, unit columns)."""
    m = T.shape[1]
    G = Y.T @ Y + EPS_LS * np.eye(Y.shape[1])
    C = np.linalg.solve(G, Y.T @ T)
    R = T - Y @ C
    L = (np.sum(R * R) + EPS_LS * np.sum(C * C)) / m
    return L, -2.0 * (R @ C.T) / m


def loss_and_grad(theta, X, targets, round_weights=True):
    """Mean loss over the batch and its gradient.  targets: list of (GRID^2, m_s)."""
    y, cache = forward(theta, X, round_weights)
    Y = vectors(y)
    S = X.shape[0]
    dY = np.zeros_like(Y)
    total = 0.0
    for s in range(S):
        L, g = sample_loss(Y[s], targets[s])
        total += L
        dY[s] = g
    dy = dY.transpose(0, 2, 1).reshape(S, OUT) / S
    return total / S, backward(cache, dy)


def unit_columns(T):
    n = np.linalg.norm(T, axis=0)
    return T / np.where(n > 0, n, 1.0)


def bilinear(Gv, u, v):
    """Values at points (u, v) in [0,1]^2 of grid vectors Gv (GRID^2, k), node
    (gx, gy) at (gx, gy) / (GRID - 1), gx fastest."""
    Gv = Gv.reshape(GRID, GRID, -1)                      # [gy][gx][k]
    s = GRID - 1
    fx, fy = np.asarray(u) * s, np.asarray(v) * s
    ix = np.minimum(np.floor(fx).astype(int), s - 1)
    iy = np.minimum(np.floor(fy).astype(int), s - 1)
    tx, ty = (fx - ix)[:, None], (fy - iy)[:, None]
    return ((1 - tx) * (1 - ty) * Gv[iy, ix] + tx * (1 - ty) * Gv[iy, ix + 1]
            + (1 - tx) * ty * Gv[iy + 1, ix] + tx * ty * Gv[iy + 1, ix + 1])


def to_nodes(Gv, nx, ny):
    """Grid vectors -> values at the nx x ny nodes of a box (x fastest)."""
    u = np.tile(np.arange(nx) / max(nx - 1, 1), ny)
    v = np.repeat(np.arange(ny) / max(ny - 1, 1), nx)
    return bilinear(Gv, u, v)


def to_grid(Wn, nx, ny):
    """Node vectors of an nx x ny box (x fastest) sampled at the GRID x GRID
    points by bilinear interpolation of the node grid."""
    V = Wn.reshape(ny, nx, -1)
    g = np.arange(GRID) / (GRID - 1)
    fx, fy = g * (nx - 1), g * (ny - 1)
    ix = np.minimum(np.floor(fx).astype(int), max(nx - 2, 0))
    iy = np.minimum(np.floor(fy).astype(int), max(ny - 2, 0))
    tx, ty = fx - ix, fy - iy
    out = np.zeros((GRID, GRID, V.shape[2]))
    for a in range(GRID):
        for b in range(GRID):
            y0, x0 = iy[a], ix[b]
            out[a, b] = ((1 - tx[b]) * (1 - ty[a]) * V[y0, x0] + tx[b] * (1 - ty[a]) * V[y0, x0 + 1]
                         + (1 - tx[b]) * ty[a] * V[y0 + 1, x0] + tx[b] * ty[a] * V[y0 + 1, x0 + 1])
    return out.reshape(GRID * GRID, -1)


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t >= 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
