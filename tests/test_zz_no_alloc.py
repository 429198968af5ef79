"""msdd_band_solve_noalloc: the band solve that allocates no device memory.

Some callers cannot let a library allocate device memory during a call: an
application that runs under a fixed memory budget or hands out all device
memory from its own pool, or a tight loop in which a cudaMalloc/cudaFree would
synchronise the device and stall its other streams.  For them the staging
buffer of the batched band solve lives in a static 16 MiB device array.

The tests call the new entry point through the C ABI twice in a row and
compare each result with the allocating msdd_band_solve: within 1e-10
relative with FP64 factors (the band-solver tolerance of the parity tests)
and within 1e-5 with FP32 factors, whose 16-column solves take the
TMA-fed band kernel.  After a first call, a further call must leave the
device's free memory unchanged.  This file is collected last so that a run
stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

import paper_2106_06404_gb300 as pkg  # noqa: E402

TOL = {0: 1e-10, 1: 1e-5}


def _batch(sizes, bw, seed):
    rng = np.random.default_rng(seed)
    nmax = max(sizes)
    A = np.zeros((len(sizes), nmax, nmax))
    for i, n in enumerate(sizes):
        M = rng.standard_normal((n, n))
        band = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= bw
        S = np.where(band, M + M.T, 0.0)
        S += np.diag(np.abs(S).sum(axis=1) + 1.0)
        A[i, :n, :n] = S
    return A


@pytest.mark.parametrize("precision,nrhs,bw", [(0, 1, 40), (0, 3, 40), (1, 16, 40), (1, 16, 60)])
def test_noalloc_matches_allocating_solve_twice(precision, nrhs, bw):
    sizes = [1, 31, 33, 64, 157, 300]
    A = _batch(sizes, bw, seed=5)
    bb = pkg.BandBatch(torch.tensor(A, device="cuda"), sizes, bw, precision=precision)
    rng = np.random.default_rng(9)
    for call in range(2):
        B = torch.tensor(rng.standard_normal((len(sizes), max(sizes), nrhs)), device="cuda")
        ref = B.clone()
        bb.solve(ref)
        out = B.clone()
        bb.solve_noalloc(out)
        ref, out = ref.cpu().numpy(), out.cpu().numpy()
        for i, n in enumerate(sizes):
            err = np.linalg.norm(out[i, :n] - ref[i, :n]) / np.linalg.norm(ref[i, :n])
            assert err <= TOL[precision], (call, n, err)
            # rows beyond n[i] are not touched
            assert np.array_equal(out[i, n:], B[i, n:].cpu().numpy())
    bb.close()


def test_noalloc_call_leaves_free_device_memory_unchanged():
    sizes = [64, 157, 300]
    A = _batch(sizes, 40, seed=3)
    bb = pkg.BandBatch(torch.tensor(A, device="cuda"), sizes, 40, precision=1)
    X = torch.ones((len(sizes), max(sizes), 16), dtype=torch.float64, device="cuda")
    bb.solve_noalloc(X)                      # first call: loads the static array
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    bb.solve_noalloc(X)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    bb.close()


def test_noalloc_rejects_batches_beyond_the_static_limit():
    sizes = [32] * 2100                       # 2100 * 32 padded rows * 32 rhs > 2^21
    A = _batch([32], 4, seed=1)[0]
    At = torch.tensor(np.broadcast_to(A, (len(sizes), 32, 32)).copy(), device="cuda")
    bb = pkg.BandBatch(At, sizes, 4, precision=0)
    X = torch.ones((len(sizes), 32, 32), dtype=torch.float64, device="cuda")
    with pytest.raises(pkg.MsddError) as e:
        bb.solve_noalloc(X)
    assert e.value.status == -1 and "static limit" in str(e.value)
    assert torch.all(X == 1.0)
    bb.close()
