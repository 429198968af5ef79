"""The integer-pipe FP64 <-> FP32 conversions that every FP32 kernel of the
library uses (f64_to_f32 / f32_to_f64, written from the IEEE 754 formats),
bit for bit against CUDA's own conversions (__double2float_rn and the float
to double widening) on edge values: signed zeros, infinities, NaN, rounding
ties at every scale, the overflow threshold, the normal/subnormal boundary,
subnormal results and inputs, and random bit patterns.  NaN results are
compared as "both NaN".

Also the double-float helpers of the chosen form's Gram products: split_f64
reconstructs x as hi + lo to 2^-47 relative (hi exact in FP32, |lo| <=
2^-23 |hi|) inside its range and falls back to (f64_to_f32(x), 0) outside,
and df_fma dot products of 1369 terms agree with the exact dot product (the
products summed as fractions) to 1e-11 of the sum of |terms|: each step adds
at most ~2^-46 of its product and the FP32 low-order sum grows by n 2^-24 of
its size, so n 2^-47 ~ 1e-11 bounds the error (measured ~1e-13)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a GPU", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2106_06404_gb300", "csrc")


@pytest.fixture(scope="module")
def probe(tmp_path_factory):
    out = str(tmp_path_factory.mktemp("conv") / "libconv.so")
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17", "-shared",
                           "-Xcompiler", "-fPIC", "-I", CSRC, "-I", os.path.join(os.path.dirname(HERE), "include"),
                           os.path.join(HERE, "fp_conversions.cu"), "-o", out])
    lib = ctypes.CDLL(out)
    lib.conv_probe.restype = ctypes.c_int
    lib.conv_probe.argtypes = [ctypes.c_void_p] * 2 + [ctypes.c_int] + [ctypes.c_void_p] * 4
    lib.df_probe.restype = ctypes.c_int
    lib.df_probe.argtypes = [ctypes.c_void_p, ctypes.c_int] + [ctypes.c_void_p] * 4 + [ctypes.c_int] * 2 + \
        [ctypes.c_void_p]
    return lib


def _edge_doubles():
    f = np.float64
    tiny, fmax = float(np.finfo(np.float32).tiny), float(np.finfo(np.float32).max)
    sub = 2.0 ** -149
    v = [0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, -1.0, tiny, -tiny, tiny * (1 - 2.0 ** -24),
         tiny * (1 - 2.0 ** -25), tiny * (1 - 2.0 ** -23), sub, sub / 2, sub * 1.5, sub * 2.5, sub * 3,
         sub * 0.49, sub * 0.51, -sub / 2, fmax, fmax * (1 + 2.0 ** -25), fmax * (1 + 2.0 ** -24),
         fmax * (1 + 2.0 ** -23), 1e39, -1e39, 1e-46, 5e-324, 2.0 ** -1022, 1 + 2.0 ** -24, 1 + 3 * 2.0 ** -24,
         1 + 2.0 ** -24 + 2.0 ** -52, 1 - 2.0 ** -25]
    rng = np.random.default_rng(0)
    # ties at random scales: float mantissa plus exactly half an ulp
    for _ in range(2000):
        e = int(rng.integers(-160, 129))
        m = int(rng.integers(0, 1 << 23))
        fl = np.ldexp(f((1 << 23) + m), e - 23)
        v += [fl + np.ldexp(1.0, e - 24), fl + np.ldexp(1.0, e - 24) * (1 + 2.0 ** -20)]
    v += list(np.exp(rng.uniform(np.log(1e-47), np.log(1e39), 20000)) * rng.choice([-1, 1], 20000))
    bits = rng.integers(0, 2 ** 63, 20000, dtype=np.int64).astype(np.uint64) | \
        (rng.integers(0, 2, 20000).astype(np.uint64) << np.uint64(63))
    v += list(bits.view(np.float64))
    return np.array(v, dtype=np.float64)


def _edge_floats():
    rng = np.random.default_rng(1)
    specials = np.array([0.0, -0.0, np.inf, -np.inf, np.nan, 1.0, np.finfo(np.float32).tiny,
                         np.finfo(np.float32).max], dtype=np.float32)
    subs = np.arange(1, 4096, dtype=np.uint32).view(np.float32)                     # smallest subnormals
    top = (np.uint32(0x007fffff) - np.arange(0, 4096, dtype=np.uint32)).view(np.float32)  # largest subnormals
    rnd = rng.integers(0, 2 ** 32, 50000, dtype=np.uint64).astype(np.uint32).view(np.float32)
    return np.concatenate([specials, subs, -subs, top, rnd])


def test_conversions_match_cuda_bit_for_bit(probe):
    xd = _edge_doubles()
    xf = _edge_floats()
    n = max(len(xd), len(xf))
    xd = np.resize(xd, n)
    xf = np.resize(xf, n)
    dev = "cuda"
    txd, txf = torch.tensor(xd, device=dev), torch.tensor(xf, device=dev)
    of, cf = torch.empty(n, dtype=torch.float32, device=dev), torch.empty(n, dtype=torch.float32, device=dev)
    od, cd = torch.empty(n, dtype=torch.float64, device=dev), torch.empty(n, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    rc = probe.conv_probe(txd.data_ptr(), txf.data_ptr(), n, of.data_ptr(), cf.data_ptr(), od.data_ptr(),
                          cd.data_ptr())
    assert rc == 0
    of, cf, od, cd = (t.cpu().numpy() for t in (of, cf, od, cd))
    bad = np.nonzero(~((of.view(np.uint32) == cf.view(np.uint32)) | (np.isnan(of) & np.isnan(cf))))[0]
    assert len(bad) == 0, [(xd[i], of[i], cf[i]) for i in bad[:5]]
    bad = np.nonzero(~((od.view(np.uint64) == cd.view(np.uint64)) | (np.isnan(od) & np.isnan(cd))))[0]
    assert len(bad) == 0, [(xf[i], od[i], cd[i]) for i in bad[:5]]
    # the host's IEEE conversions agree as well (numpy rounds to nearest even)
    ref = xd.astype(np.float32)
    assert np.all((of.view(np.uint32) == ref.view(np.uint32)) | (np.isnan(of) & np.isnan(ref)))


def test_double_float_split_and_dot(probe):
    from fractions import Fraction
    rng = np.random.default_rng(7)
    x = np.exp(rng.uniform(np.log(2.0 ** -59), np.log(2.0 ** 99), 20000)) * rng.choice([-1, 1], 20000)
    x = np.concatenate([x, [0.0, -0.0, 1.0, -1.0, 2.0 ** -70, 3.0 ** 70, 1e-300, 1 + 2.0 ** -52]])
    rows, L = 64, 1369
    a = rng.standard_normal((rows, L)) * np.exp(rng.uniform(-20, 20, (rows, 1)))
    b = rng.standard_normal((rows, L)) * np.exp(rng.uniform(-20, 20, (rows, 1)))
    dev = "cuda"
    tx, ta, tb = (torch.tensor(v, device=dev) for v in (x, a, b))
    hi = torch.empty(len(x), dtype=torch.float32, device=dev)
    lo = torch.empty(len(x), dtype=torch.float32, device=dev)
    dot = torch.empty(rows, dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    assert probe.df_probe(tx.data_ptr(), len(x), hi.data_ptr(), lo.data_ptr(), ta.data_ptr(), tb.data_ptr(), rows, L,
                          dot.data_ptr()) == 0
    hi, lo, dot = hi.cpu().numpy(), lo.cpu().numpy(), dot.cpu().numpy()
    inside = (np.abs(x) >= 2.0 ** -60) & (np.abs(x) < 2.0 ** 101)
    rec = hi.astype(np.float64) + lo.astype(np.float64)
    assert np.all(np.abs(x - rec)[inside] <= 2.0 ** -47 * np.abs(x[inside]))
    assert np.all(np.abs(lo[inside].astype(np.float64)) <= 2.0 ** -23 * np.abs(hi[inside].astype(np.float64)))
    assert np.all(hi[~inside] == x[~inside].astype(np.float32)) and np.all(lo[~inside] == 0)
    worst = 0.0
    for r in range(rows):
        exact = float(sum((Fraction(u) * Fraction(v) for u, v in zip(a[r], b[r])), Fraction(0)))
        scale = float(np.sum(np.abs(a[r] * b[r])))
        worst = max(worst, abs(dot[r] - exact) / scale)
    print("double-float dot products: max error %.2e of the sum of |terms|" % worst)
    assert worst <= 1e-11
