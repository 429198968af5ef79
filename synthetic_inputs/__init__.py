"""Seeded synthetic coefficient fields and workload descriptions.

The one module that both the CUDA path's callers (tests, bench.py) and the CPU
oracle use.  It generates inputs only (numpy PCG64 streams); it holds none of
the method's arithmetic.

The paper's own data (the "islands" field of Section 5.1, SPE10 of Section
5.2, the composite geometry of Section 5.3) are not available; the fields
below stand in for their structure: isolated or channelised high-conductivity
regions with contrast up to 1e6, a log-normal background, and layered
anisotropic tensors.

Element arrays are flat, element (ex, ey[, ez]) at ex + nx * (ey + ny * ez).
"""
from dataclasses import dataclass, field
from typing import Optional, Tuple

import numpy as np


def channels_2d(N, n_channels=8, contrast=1e6, seed=0):
    """kappa = 1 with `n_channels` one-element-high horizontal channels of kappa = contrast.

    Channel rows are rng.choice(N, n_channels, replace=False) with PCG64(seed).
    """
    rng = np.random.default_rng(seed)
    rows = rng.choice(N, n_channels, replace=False)
    k = np.ones((N, N))
    k[rows, :] = contrast
    return k.ravel()


def gaussian_random_field_2d(N, corr_len=0.05, variance=2.0, rng=None):
    """Stationary Gaussian field at element centres of an N x N grid on [0,1]^2.

    Exponential covariance variance * exp(-r / corr_len), sampled exactly by
    circulant embedding on a 2N x 2N periodic grid (spacing 1/N); negative
    eigenvalues of the embedding, if any, are clipped to zero.
    Returns (field (N*N,), number of clipped eigenvalues).
    """
    rng = rng if rng is not None else np.random.default_rng(0)
    M = 2 * N
    h = 1.0 / N
    idx = np.arange(M)
    d = np.minimum(idx, M - idx) * h                      # periodic distance
    r = np.sqrt(d[:, None] ** 2 + d[None, :] ** 2)
    c = variance * np.exp(-r / corr_len)
    lam = np.fft.fft2(c).real
    clipped = int(np.sum(lam < 0))
    lam = np.maximum(lam, 0.0)
    eps = rng.standard_normal((M, M)) + 1j * rng.standard_normal((M, M))
    y = np.fft.fft2(np.sqrt(lam / (M * M)) * eps)
    return y.real[:N, :N].ravel(), clipped


def grf_channels_inclusions_2d(N, seed=0, corr_len=0.05, variance=2.0, contrast=1e6,
                               n_channels=16, channel_width=2, n_inclusions=32,
                               inclusion_side=(8, 24)):
    """exp(GRF) multiplied by `contrast` on seeded channels and square inclusions."""
    rng = np.random.default_rng(seed)
    g, _ = gaussian_random_field_2d(N, corr_len, variance, rng)
    k = np.exp(g).reshape(N, N)
    mask = np.zeros((N, N), dtype=bool)
    starts = rng.choice(N - channel_width + 1, n_channels, replace=False)
    for s in starts:
        mask[s:s + channel_width, :] = True
    for _ in range(n_inclusions):
        side = int(rng.integers(inclusion_side[0], inclusion_side[1] + 1))
        x0 = int(rng.integers(0, N - side + 1))
        y0 = int(rng.integers(0, N - side + 1))
        mask[y0:y0 + side, x0:x0 + side] = True
    k[mask] *= contrast
    return k.ravel()


def composite_3d(N, seed=0, ply_aniso=1e-3, resin=1e-2, n_ply=9, n_resin=8, resin_thickness=2):
    """Layered anisotropic tensor field on an N^3 grid (kxx, kyy, kzz, kyz, kxz, kxy).

    Layers stacked in z: plies (diag(1, a, a) rotated by +-45 degrees about z,
    alternating sign from a seeded start) separated by resin layers
    (resin * I) of `resin_thickness` elements; ply thicknesses are near-equal
    and sum with the resin layers to N (seeded assignment of the remainder).
    """
    rng = np.random.default_rng(seed)
    ply_total = N - n_resin * resin_thickness
    base, rem = divmod(ply_total, n_ply)
    thick = np.full(n_ply, base)
    thick[rng.choice(n_ply, rem, replace=False)] += 1
    sign = 1.0 if rng.integers(0, 2) else -1.0
    comps = np.zeros((N, N, N, 6))                         # [z, y, x, c]
    z = 0
    for p in range(n_ply):
        th = sign * np.pi / 4.0
        c, s = np.cos(th), np.sin(th)
        R = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
        K = R @ np.diag([1.0, ply_aniso, ply_aniso]) @ R.T
        comps[z:z + thick[p], :, :, :] = [K[0, 0], K[1, 1], K[2, 2], K[1, 2], K[0, 2], K[0, 1]]
        z += thick[p]
        sign = -sign
        if p < n_resin:
            comps[z:z + resin_thickness, :, :, :] = [resin, resin, resin, 0.0, 0.0, 0.0]
            z += resin_thickness
    assert z == N
    return comps.reshape(N * N * N, 6)


def rotated_channels_2d(N, n_channels=4, contrast=1e4, aniso=1e-2, seed=0):
    """Seeded 2D tensor field (kxx, kyy, kxy) per element: the scalar field
    channels_2d(N, n_channels, contrast, seed) times R diag(1, aniso) R^T, R
    the rotation by an angle drawn uniformly from [0, pi) per element
    (PCG64(seed + 1)); element-major, x fastest."""
    k = channels_2d(N, n_channels, contrast, seed)
    th = np.random.default_rng(seed + 1).uniform(0.0, np.pi, N * N)
    c, s = np.cos(th), np.sin(th)
    return np.stack([k * (c * c + aniso * s * s), k * (s * s + aniso * c * c), k * (1.0 - aniso) * c * s], axis=1)


def layered_3d(N, seed=0, contrast=1e4):
    """Seeded 3D scalar field for small 3D cases: one-element layers along z
    alternating kappa 1 and `contrast`, times exp(0.5 g) with g standard normal
    per element (PCG64(seed)); element-major, x fastest."""
    rng = np.random.default_rng(seed)
    z = np.arange(N)
    layer = np.where(z % 2 == 0, 1.0, contrast)
    k = layer[:, None, None] * np.ones((N, N, N)) * np.exp(0.5 * rng.standard_normal((N, N, N)))
    return k.ravel()


@dataclass
class Workload:
    """A named problem: mesh, coefficient recipe, decomposition, spectral options."""
    name: str
    n: Tuple[int, ...]
    parts: Tuple[int, ...]
    overlap: int
    levels: int
    group: Tuple[int, ...]
    nev_max: int
    eta: float
    dirichlet_faces: int = 0b1
    seed: int = 0
    kind: str = "channels"
    contrast: float = 1e6
    extra: dict = field(default_factory=dict)

    def coefficient(self):
        if self.kind == "channels":
            return channels_2d(self.n[0], self.extra.get("n_channels", 8), self.contrast, self.seed)
        if self.kind == "grf":
            return grf_channels_inclusions_2d(self.n[0], self.seed, contrast=self.contrast, **self.extra)
        if self.kind == "composite":
            return composite_3d(self.n[0], self.seed)
        if self.kind == "constant":
            return np.ones(int(np.prod(self.n)))
        raise ValueError(self.kind)


def channels64(seed=0, contrast=1e6):
    """2D, 64 x 64 Q1, 8 channels, 4 x 4 subdomains, overlap 2, two levels, nev <= 8."""
    return Workload("channels2d_64x64_4x4_2lvl", (64, 64), (4, 4), 2, 2, (4, 4), 8, 0.3,
                    seed=seed, kind="channels", contrast=contrast)


def grf512(seed=0):
    """2D, 512 x 512 Q1, GRF x channels/inclusions 1e6, 16 x 16 subdomains, three levels, nev <= 12."""
    return Workload("grf2d_512x512_16x16_3lvl", (512, 512), (16, 16), 2, 3, (4, 4), 12, 0.3,
                    seed=seed, kind="grf")


def composite128(seed=0):
    """3D, 128^3 Q1, layered anisotropic tensor, 8^3 subdomains, overlap 1, three levels, nev <= 16."""
    return Workload("composite3d_128_8x8x8_3lvl", (128, 128, 128), (8, 8, 8), 1, 3, (2, 2, 2), 16, 0.3,
                    seed=seed, kind="composite")


def composite96(seed=0):
    """3D, 96^3 Q1, the layered composite of composite128 at 6^3 subdomains, overlap 1, three levels,
    nev <= 16: the same box shapes as the 128^3 workload's Dirichlet matrices (16^3 elements per
    subdomain) at a size small enough for a full ncu capture."""
    return Workload("composite3d_96_6x6x6_3lvl", (96, 96, 96), (6, 6, 6), 1, 3, (2, 2, 2), 16, 0.3,
                    seed=seed, kind="composite")


def batch256(seed=0, count=256):
    """Batch of independent 2D problems of uneven size: per problem, from one
    PCG64(seed) stream in this order, the side N ~ U{128..384} elements, the
    subdomains per axis P ~ U{4..12}, the contrast 10^U[4, 6] and the field
    seed.  Coefficient: exp(GRF) (correlation length 0.05, variance 2) times
    the contrast on N // 16 one-element channels, no inclusions.  Two levels,
    overlap 2, nev <= 8, eta = 0.3, Dirichlet on x = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        N = int(rng.integers(128, 385))
        P = int(rng.integers(4, 13))
        contrast = float(10.0 ** rng.uniform(4.0, 6.0))
        fseed = int(rng.integers(0, 2**31 - 1))
        out.append(Workload("batch2d_%03d_%dx%d_%dx%d" % (i, N, N, P, P), (N, N), (P, P), 2, 2, (1, 1), 8, 0.3,
                            seed=fseed, kind="grf", contrast=contrast,
                            extra={"n_channels": N // 16, "channel_width": 1, "n_inclusions": 0}))
    return out


def mlp_init(seed, shapes):
    """Seeded He-normal weights (std sqrt(2 / fan_in) for 2-D shapes (fan_out, fan_in)),
    zero biases (1-D shapes), concatenated row-major as float32."""
    rng = np.random.default_rng(seed)
    parts = []
    for s in shapes:
        if len(s) == 2:
            parts.append(rng.standard_normal(s) * np.sqrt(2.0 / s[1]))
        else:
            parts.append(np.zeros(s))
    return np.concatenate([p.ravel() for p in parts]).astype(np.float32)
