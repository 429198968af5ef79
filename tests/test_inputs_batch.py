"""Input recipes: the batched multi-problem recipe (256 seeded 2D problems of
uneven size: sides 128..384, 4x4..12x12 subdomains, contrast 1e4..1e6) and
the 2D tensor field of the tensor-coefficient parity cases."""
import numpy as np

import synthetic_inputs as si


def test_batch_recipe_ranges_and_determinism():
    b = si.batch256(seed=0)
    assert len(b) == 256
    sides = np.array([w.n[0] for w in b])
    parts = np.array([w.parts[0] for w in b])
    contrast = np.array([w.contrast for w in b])
    assert all(w.n[0] == w.n[1] and w.parts[0] == w.parts[1] for w in b)
    assert sides.min() >= 128 and sides.max() <= 384 and sides.max() - sides.min() > 200
    assert parts.min() == 4 and parts.max() == 12
    assert contrast.min() >= 1e4 and contrast.max() <= 1e6
    assert np.log10(contrast).std() > 0.4                 # spread over the two decades
    assert len({w.seed for w in b}) == 256
    again = si.batch256(seed=0)
    assert [(w.n, w.parts, w.contrast, w.seed) for w in again] == [(w.n, w.parts, w.contrast, w.seed) for w in b]
    assert [(w.n, w.seed) for w in si.batch256(seed=1)] != [(w.n, w.seed) for w in b]


def test_batch_coefficients():
    for w in si.batch256(seed=0, count=4):
        k = w.coefficient()
        N = w.n[0]
        assert k.shape == (N * N,) and np.all(k > 0) and np.all(np.isfinite(k))
        rows = k.reshape(N, N)
        # the channel rows carry the contrast on top of the log-normal background
        ratio = np.exp(np.median(np.log(rows), axis=1))
        assert np.sum(ratio > np.sqrt(w.contrast)) == N // 16


def test_rotated_channel_tensors():
    """The 2D tensor field: per element a symmetric tensor with eigenvalues
    k and aniso * k, k the channel field's value; seeded."""
    N, aniso = 20, 1e-2
    T = si.rotated_channels_2d(N, n_channels=3, contrast=1e4, aniso=aniso, seed=5)
    k = si.channels_2d(N, 3, 1e4, seed=5)
    assert T.shape == (N * N, 3)
    M = np.stack([np.stack([T[:, 0], T[:, 2]], 1), np.stack([T[:, 2], T[:, 1]], 1)], 1)
    ev = np.linalg.eigvalsh(M)
    assert np.allclose(ev[:, 0], aniso * k, rtol=1e-12) and np.allclose(ev[:, 1], k, rtol=1e-12)
    assert np.array_equal(T, si.rotated_channels_2d(N, n_channels=3, contrast=1e4, aniso=aniso, seed=5))
