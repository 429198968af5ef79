"""Thin ctypes binding of the msdd C ABI (include/msdd.h).

Argument marshalling only: every step runs in the CUDA library.  PyTorch
provides device memory (CUDA tensors) and the current stream.  There is no
CPU fallback: if the library is missing or no GPU is present, calls fail.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libmsdd.so")

MSDD_OK = 0
STATUS_NAMES = {
    0: "MSDD_OK", -1: "MSDD_ERR_INVALID_ARG", -2: "MSDD_ERR_NOT_SPD", -3: "MSDD_ERR_NO_CONVERGENCE",
    -4: "MSDD_ERR_EIG_NO_CONVERGENCE", -5: "MSDD_ERR_OOM", -6: "MSDD_ERR_CUDA", -7: "MSDD_ERR_UNSUPPORTED",
    -8: "MSDD_ERR_TIMEOUT",
}
MAX_LEVELS = 8


class MsddError(RuntimeError):
    def __init__(self, status, message):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), message))
        self.status = status


class Mesh(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dirichlet_faces", ctypes.c_uint)]


class Coeff(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("data", ctypes.c_void_p)]


class Decomp(ctypes.Structure):
    _fields_ = [("parts", ctypes.c_int * 3), ("overlap", ctypes.c_int), ("levels", ctypes.c_int),
                ("group", ctypes.c_int * 3)]


class Spectral(ctypes.Structure):
    _fields_ = [("nev_max", ctypes.c_int), ("eta", ctypes.c_double), ("blf", ctypes.c_int)]


class Options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("block_p", ctypes.c_int), ("eig_maxit", ctypes.c_int),
                ("sigma", ctypes.c_double), ("eig_tol", ctypes.c_double), ("reg_tol", ctypes.c_double),
                ("seed", ctypes.c_ulonglong), ("stream", ctypes.c_void_p), ("profile", ctypes.c_int),
                ("fp32_start_iters", ctypes.c_int), ("warm_start", ctypes.c_void_p), ("warm_cols", ctypes.c_int)]


class KernelProf(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int), ("ms", ctypes.c_double),
                ("bytes", ctypes.c_double), ("flops", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_longlong), ("levels", ctypes.c_int), ("precision", ctypes.c_int),
                ("subdomains", ctypes.c_int * MAX_LEVELS), ("level_dim", ctypes.c_longlong * MAX_LEVELS),
                ("eig_iters_max", ctypes.c_int * MAX_LEVELS), ("eig_iters_min", ctypes.c_int * MAX_LEVELS),
                ("eig_unconverged", ctypes.c_int * MAX_LEVELS), ("eig_at_floor", ctypes.c_int * MAX_LEVELS),
                ("null_pivots", ctypes.c_int * MAX_LEVELS),
                ("m_min", ctypes.c_int * MAX_LEVELS), ("m_max", ctypes.c_int * MAX_LEVELS),
                ("setup_ms", ctypes.c_double), ("phase_ms", ctypes.c_double * 8),
                ("pcg_iterations", ctypes.c_int), ("pcg_rel_residual", ctypes.c_double),
                ("solve_ms", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("nprof", ctypes.c_int), ("prof", KernelProf * 12),
                ("eig_iters_total", ctypes.c_longlong * MAX_LEVELS)]


EXPORTED = [
    "msdd_default_options", "msdd_num_unknowns", "msdd_setup", "msdd_solve", "msdd_solve_host",
    "msdd_apply_preconditioner", "msdd_apply_operator", "msdd_assemble_rhs", "msdd_get_stats",
    "msdd_get_eigenvalues", "msdd_get_eigen_residuals", "msdd_get_fine_basis", "msdd_destroy", "msdd_last_error",
    "msdd_band_factor", "msdd_band_solve", "msdd_band_destroy", "msdd_band_solve_noalloc", "msdd_kernel_launches",
    "msdd_fine_layout", "msdd_nn_patches", "msdd_nn_workspace_bytes", "msdd_nn_forward", "msdd_nn_loss_grad",
    "msdd_nn_adam", "msdd_nn_start_vectors", "msdd_nn_targets", "msdd_release_cache", "msdd_cached_bytes",
    "msdd_apply_hybrid_preconditioner", "msdd_solve_gmres", "msdd_batch_plan", "msdd_batch_run",
]

# learned warm start (include/msdd.h, MSDD_NN_*)
NN_PATCH, NN_HIDDEN, NN_GRID, NN_NVEC = 24, 48, 13, 12
NN_IN, NN_OUT = NN_PATCH * NN_PATCH, NN_NVEC * NN_GRID * NN_GRID
NN_NPARAM = NN_HIDDEN * NN_IN + NN_HIDDEN + NN_HIDDEN * NN_HIDDEN + NN_HIDDEN + NN_OUT * NN_HIDDEN + NN_OUT

_lib = None


def load(path=LIB_PATH):
    """Load libmsdd.so (raises OSError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise OSError("libmsdd.so not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp, dp, ip = ctypes.c_void_p, P(ctypes.c_double), P(ctypes.c_int)
    lib.msdd_default_options.argtypes = [P(Options)]
    lib.msdd_num_unknowns.argtypes = [P(Mesh)]
    lib.msdd_num_unknowns.restype = ctypes.c_longlong
    lib.msdd_setup.argtypes = [P(Mesh), P(Coeff), P(Decomp), P(Spectral), P(Options), P(vp)]
    lib.msdd_solve.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp, ip, dp]
    lib.msdd_solve_host.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, vp, ip, dp]
    lib.msdd_apply_preconditioner.argtypes = [vp, vp, vp]
    lib.msdd_apply_hybrid_preconditioner.argtypes = [vp, vp, vp]
    lib.msdd_solve_gmres.argtypes = [vp, vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, vp, ip, dp]
    lib.msdd_apply_operator.argtypes = [vp, vp, vp]
    lib.msdd_assemble_rhs.argtypes = [P(Mesh), ctypes.c_double, vp, vp]
    lib.msdd_get_stats.argtypes = [vp, P(Stats)]
    lib.msdd_get_eigenvalues.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip, ip]
    lib.msdd_get_eigen_residuals.argtypes = [vp, ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ip]
    lib.msdd_get_fine_basis.argtypes = [vp, ctypes.c_int, dp, ctypes.c_longlong, ip]
    lib.msdd_destroy.argtypes = [vp]
    lib.msdd_destroy.restype = None
    lib.msdd_last_error.restype = ctypes.c_char_p
    lib.msdd_band_factor.argtypes = [ctypes.c_int, ip, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                     ctypes.c_double, vp, P(vp), ip]
    lib.msdd_band_solve.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.msdd_band_solve_noalloc.argtypes = [vp, ctypes.c_int, vp, vp]
    lib.msdd_band_destroy.argtypes = [vp]
    lib.msdd_band_destroy.restype = None
    lib.msdd_kernel_launches.argtypes = []
    lib.msdd_kernel_launches.restype = ctypes.c_longlong
    lib.msdd_release_cache.argtypes = []
    lib.msdd_cached_bytes.argtypes = []
    lib.msdd_cached_bytes.restype = ctypes.c_longlong
    lib.msdd_fine_layout.argtypes = [P(Mesh), P(Decomp), ip, ctypes.c_int, ip]
    lib.msdd_batch_plan.argtypes = [ctypes.c_int, P(Mesh), P(Decomp), ctypes.c_int, ip, dp, ctypes.c_longlong,
                                    P(ctypes.c_longlong), dp, dp]
    lib.msdd_batch_run.argtypes = [ctypes.c_int, P(Mesh), P(Coeff), P(Decomp), P(Spectral), P(Options), P(vp),
                                   ctypes.c_double, ctypes.c_int, P(vp), ctypes.c_int, ip, dp, ip, dp, dp]
    lib.msdd_nn_patches.argtypes = [P(Mesh), P(Coeff), P(Decomp), vp, vp]
    lib.msdd_nn_workspace_bytes.argtypes = [ctypes.c_int]
    lib.msdd_nn_workspace_bytes.restype = ctypes.c_size_t
    lib.msdd_nn_forward.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp]
    lib.msdd_nn_loss_grad.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, vp, vp]
    lib.msdd_nn_adam.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_float, vp]
    lib.msdd_nn_start_vectors.argtypes = [P(Mesh), P(Decomp), vp, vp, vp]
    lib.msdd_nn_targets.argtypes = [vp, vp, vp, vp]
    for name in EXPORTED:
        if name in ("msdd_last_error", "msdd_destroy", "msdd_band_destroy", "msdd_num_unknowns",
                    "msdd_kernel_launches", "msdd_nn_workspace_bytes", "msdd_cached_bytes"):
            continue
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _check(status, allow=()):
    if status != MSDD_OK and status not in allow:
        raise MsddError(status, load().msdd_last_error().decode())
    return status


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("msdd needs a CUDA GPU")
    return torch


def _stream():
    torch = _torch()
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def make_mesh(n, dirichlet_faces=0b1):
    m = Mesh()
    m.dim = len(n)
    for d in range(3):
        m.n[d] = int(n[d]) if d < len(n) else 1
    m.dirichlet_faces = int(dirichlet_faces)
    return m


def num_unknowns(n, dirichlet_faces=0b1):
    return int(load().msdd_num_unknowns(ctypes.byref(make_mesh(n, dirichlet_faces))))


def assemble_rhs(n, dirichlet_faces=0b1, f=1.0):
    torch = _torch()
    mesh = make_mesh(n, dirichlet_faces)
    b = torch.empty(num_unknowns(n, dirichlet_faces), dtype=torch.float64, device="cuda")
    _check(load().msdd_assemble_rhs(ctypes.byref(mesh), float(f), ctypes.c_void_p(b.data_ptr()), _stream()))
    return b


def kernel_launches():
    """Kernels launched by the library in this process so far."""
    return int(load().msdd_kernel_launches())


def release_cache():
    """msdd_release_cache: return the library's cached device blocks to the driver."""
    _check(load().msdd_release_cache())


def cached_bytes():
    """msdd_cached_bytes: device bytes held by the library's allocation cache."""
    return int(load().msdd_cached_bytes())


def default_options():
    o = Options()
    load().msdd_default_options(ctypes.byref(o))
    return o


class Hierarchy:
    """msdd_setup / msdd_solve on CUDA tensors.

    coeff: CUDA float64 tensor, (num_elements,) scalar or (num_elements, 3|6) tensor.
    """

    def __init__(self, n, coeff, parts, overlap, levels, group, nev_max, eta, dirichlet_faces=0b1,
                 precision=0, block_p=0, eig_maxit=200, sigma=1e-2, eig_tol=1e-6, reg_tol=-1.0, seed=12345,
                 allow_eig_unconverged=False, profile=False, fp32_start_iters=None, warm_start=None, blf=1):
        torch = _torch()
        lib = load()
        self._lib = lib
        self.mesh = make_mesh(n, dirichlet_faces)
        coeff = coeff.to(device="cuda", dtype=torch.float64).contiguous()
        self._coeff = coeff                      # alive until msdd_setup has copied it
        c = Coeff()
        c.kind = 0 if coeff.dim() == 1 else 1
        c.data = coeff.data_ptr()
        d = Decomp()
        for k in range(3):
            d.parts[k] = int(parts[k]) if k < len(parts) else 1
            d.group[k] = int(group[k]) if k < len(group) else 1
        d.overlap = int(overlap)
        d.levels = int(levels)
        s = Spectral()
        s.nev_max = int(nev_max)
        s.eta = float(eta)
        s.blf = int(blf)
        o = default_options()
        o.precision, o.block_p, o.eig_maxit = int(precision), int(block_p), int(eig_maxit)
        o.sigma, o.eig_tol, o.reg_tol, o.seed = float(sigma), float(eig_tol), float(reg_tol), int(seed)
        o.stream = torch.cuda.current_stream().cuda_stream
        o.profile = 2 if profile == 2 else (1 if profile else 0)
        if fp32_start_iters is not None:
            o.fp32_start_iters = int(fp32_start_iters)
        if warm_start is not None:
            # start vectors of the fine subspace iteration: rows as fine_layout(), float64 CUDA
            warm_start = warm_start.to(device="cuda", dtype=torch.float64).contiguous()
            o.warm_start = warm_start.data_ptr()
            o.warm_cols = int(warm_start.shape[1])
        h = ctypes.c_void_p()
        st = lib.msdd_setup(ctypes.byref(self.mesh), ctypes.byref(c), ctypes.byref(d), ctypes.byref(s),
                            ctypes.byref(o), ctypes.byref(h))
        self.setup_status = st
        _check(st, allow=(-4,) if allow_eig_unconverged else ())
        self._h = h
        self.n = num_unknowns(n, dirichlet_faces)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msdd_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, tol=1e-8, maxit=1000, out=None, allow_maxit=False):
        torch = _torch()
        x = out if out is not None else torch.empty_like(b)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        st = self._lib.msdd_solve(self._h, ctypes.c_void_p(b.data_ptr()), float(tol), int(maxit),
                                  ctypes.c_void_p(x.data_ptr()), ctypes.byref(it), ctypes.byref(rel))
        _check(st, allow=(-3,) if allow_maxit else ())
        return x, it.value, rel.value

    def solve_gmres(self, b, tol=1e-8, restart=200, maxit=1000, allow_maxit=False):
        """msdd_solve_gmres: GMRES with the hybrid preconditioner (x0 = 0)."""
        torch = _torch()
        x = torch.empty_like(b)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        st = self._lib.msdd_solve_gmres(self._h, ctypes.c_void_p(b.data_ptr()), float(tol), int(restart), int(maxit),
                                        ctypes.c_void_p(x.data_ptr()), ctypes.byref(it), ctypes.byref(rel))
        _check(st, allow=(-3,) if allow_maxit else ())
        return x, it.value, rel.value

    def apply_hybrid(self, r):
        """msdd_apply_hybrid_preconditioner: z = B_h r."""
        torch = _torch()
        z = torch.empty_like(r)
        _check(self._lib.msdd_apply_hybrid_preconditioner(self._h, ctypes.c_void_p(r.data_ptr()),
                                                          ctypes.c_void_p(z.data_ptr())))
        return z

    def solve_host(self, b, tol=1e-8, maxit=1000):
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.empty_like(b)
        it = ctypes.c_int()
        rel = ctypes.c_double()
        _check(self._lib.msdd_solve_host(self._h, ctypes.c_void_p(b.ctypes.data), float(tol), int(maxit),
                                         ctypes.c_void_p(x.ctypes.data), ctypes.byref(it), ctypes.byref(rel)))
        return x, it.value, rel.value

    def apply_preconditioner(self, r):
        torch = _torch()
        z = torch.empty_like(r)
        _check(self._lib.msdd_apply_preconditioner(self._h, ctypes.c_void_p(r.data_ptr()),
                                                   ctypes.c_void_p(z.data_ptr())))
        return z

    def apply_operator(self, x):
        torch = _torch()
        y = torch.empty_like(x)
        _check(self._lib.msdd_apply_operator(self._h, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(y.data_ptr())))
        return y

    def stats(self):
        s = Stats()
        _check(self._lib.msdd_get_stats(self._h, ctypes.byref(s)))
        lv = s.levels
        return {
            "n": s.n, "levels": lv, "precision": s.precision,
            "subdomains": list(s.subdomains[:lv]), "level_dim": list(s.level_dim[:lv]),
            "eig_iters_max": list(s.eig_iters_max[:lv]), "eig_iters_min": list(s.eig_iters_min[:lv]),
            "eig_iters_total": list(s.eig_iters_total[:lv]),
            "eig_unconverged": list(s.eig_unconverged[:lv]), "eig_at_floor": list(s.eig_at_floor[:lv]),
            "null_pivots": list(s.null_pivots[:lv]),
            "m_min": list(s.m_min[:lv]), "m_max": list(s.m_max[:lv]),
            "setup_ms": s.setup_ms, "phase_ms": list(s.phase_ms),
            "pcg_iterations": s.pcg_iterations, "pcg_rel_residual": s.pcg_rel_residual,
            "solve_ms": s.solve_ms, "device_bytes": s.device_bytes,
            "prof": {s.prof[k].name.decode(): dict(launches=s.prof[k].launches, ms=s.prof[k].ms,
                                                   bytes=s.prof[k].bytes, flops=s.prof[k].flops)
                     for k in range(s.nprof)},
        }

    def eigenvalues(self, level, subdomain):
        out = (ctypes.c_double * 32)()
        cnt, sel = ctypes.c_int(), ctypes.c_int()
        _check(self._lib.msdd_get_eigenvalues(self._h, int(level), int(subdomain), out, 32, ctypes.byref(cnt),
                                              ctypes.byref(sel)))
        return np.array(out[:cnt.value]), sel.value

    def eigen_residuals(self, level, subdomain):
        out = (ctypes.c_double * 32)()
        conv = ctypes.c_int()
        _check(self._lib.msdd_get_eigen_residuals(self._h, int(level), int(subdomain), out, 32, ctypes.byref(conv)))
        theta, _ = self.eigenvalues(level, subdomain)
        return np.array(out[:len(theta)]), bool(conv.value)

    def nn_targets(self):
        """Training targets of the warm-start network from this hierarchy's fine
        eigenvectors: (T float32 (P, NVEC, GRID^2), m int32 (P,)) on the GPU."""
        torch = _torch()
        P = self.stats()["subdomains"][-1]
        T = torch.empty((P, NN_NVEC, NN_GRID * NN_GRID), dtype=torch.float32, device="cuda")
        m = torch.empty(P, dtype=torch.int32, device="cuda")
        _check(self._lib.msdd_nn_targets(self._h, ctypes.c_void_p(T.data_ptr()), ctypes.c_void_p(m.data_ptr()),
                                         _stream()))
        return T, m

    def fine_basis(self, subdomain, m_max=32):
        buf = np.zeros(self.n * m_max)
        m = ctypes.c_int()
        _check(self._lib.msdd_get_fine_basis(self._h, int(subdomain), buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                             buf.size, ctypes.byref(m)))
        return buf[: self.n * m.value].reshape(self.n, m.value)


class BandBatch:
    """msdd_band_factor / msdd_band_solve: batched banded SPD LDL^T."""

    def __init__(self, A, n, bw, precision=0, reg_tol=0.0):
        torch = _torch()
        lib = load()
        self._lib = lib
        A = A.to(device="cuda", dtype=torch.float64).contiguous()
        self.batch, self.nmax = A.shape[0], A.shape[1]
        nv = (ctypes.c_int * self.batch)(*[int(v) for v in n])
        status = (ctypes.c_int * self.batch)()
        h = ctypes.c_void_p()
        st = lib.msdd_band_factor(self.batch, nv, self.nmax, int(bw), ctypes.c_void_p(A.data_ptr()), int(precision),
                                  float(reg_tol), _stream(), ctypes.byref(h), status)
        self.status = list(status)
        _check(st)
        self._h = h

    def solve(self, X):
        """Solve in place: X is (batch, nmax, nrhs) float64 CUDA."""
        _check(self._lib.msdd_band_solve(self._h, X.shape[2], ctypes.c_void_p(X.data_ptr()), _stream()))
        return X

    def solve_noalloc(self, X):
        """Same as solve() through msdd_band_solve_noalloc: no device allocation in the call
        (static 16 MiB staging array; overlapping calls must be serialised)."""
        _check(self._lib.msdd_band_solve_noalloc(self._h, X.shape[2], ctypes.c_void_p(X.data_ptr()), _stream()))
        return X

    def close(self):
        if getattr(self, "_h", None):
            self._lib.msdd_band_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _decomp(parts, overlap):
    d = Decomp()
    for k in range(3):
        d.parts[k] = int(parts[k]) if k < len(parts) else 1
        d.group[k] = 1
    d.overlap = int(overlap)
    d.levels = 2
    return d


def batch_plan(problems, nworkers):
    """msdd_batch_plan for a list of (n, parts, overlap, dirichlet_faces):
    returns (items (K, 2) int32 of (problem, subdomain) in queue order,
    costs (K,), makespan, lower_bound)."""
    lib = load()
    k = len(problems)
    meshes, decs = (Mesh * k)(), (Decomp * k)()
    for i, (n, parts, overlap, faces) in enumerate(problems):
        meshes[i] = make_mesh(n, faces)
        decs[i] = _decomp(parts, overlap)
    cnt = ctypes.c_longlong()
    _check(lib.msdd_batch_plan(k, meshes, decs, int(nworkers), None, None, 0, ctypes.byref(cnt), None, None))
    items = np.zeros(2 * cnt.value, dtype=np.int32)
    cost = np.zeros(cnt.value, dtype=np.float64)
    mk, lb = ctypes.c_double(), ctypes.c_double()
    _check(lib.msdd_batch_plan(k, meshes, decs, int(nworkers), items.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                               cost.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), cnt.value, ctypes.byref(cnt),
                               ctypes.byref(mk), ctypes.byref(lb)))
    return items.reshape(-1, 2), cost, mk.value, lb.value


def batch_run(problems, nev_max, eta, tol=1e-8, maxit=1000, precision=1, nworkers=8, allow_fail=False, **opts):
    """msdd_batch_run: set up and solve independent problems on the GPU.

    problems: list of dicts with n, kappa (CUDA float64 tensor), parts, overlap,
    levels, group, b (CUDA float64 right-hand side) and optionally
    dirichlet_faces.  Returns (xs, iterations, rel_residuals, statuses,
    setup_ms, solve_ms) with one entry per problem (xs: CUDA tensors)."""
    torch = _torch()
    lib = load()
    k = len(problems)
    meshes, coeffs, decs = (Mesh * k)(), (Coeff * k)(), (Decomp * k)()
    keep, xs = [], []
    bp, xp = (ctypes.c_void_p * k)(), (ctypes.c_void_p * k)()
    for i, pr in enumerate(problems):
        meshes[i] = make_mesh(pr["n"], pr.get("dirichlet_faces", 0b1))
        kap = pr["kappa"].to(device="cuda", dtype=torch.float64).contiguous()
        b = pr["b"].to(device="cuda", dtype=torch.float64).contiguous()
        keep += [kap, b]
        coeffs[i].kind = 0 if kap.dim() == 1 else 1
        coeffs[i].data = kap.data_ptr()
        d = Decomp()
        for a in range(3):
            d.parts[a] = int(pr["parts"][a]) if a < len(pr["parts"]) else 1
            g = pr.get("group", (1, 1, 1))
            d.group[a] = int(g[a]) if a < len(g) else 1
        d.overlap = int(pr["overlap"])
        d.levels = int(pr.get("levels", 2))
        decs[i] = d
        x = torch.zeros_like(b)
        xs.append(x)
        bp[i], xp[i] = b.data_ptr(), x.data_ptr()
    s = Spectral()
    s.nev_max, s.eta, s.blf = int(nev_max), float(eta), 1
    o = default_options()
    o.precision = int(precision)
    for key, val in opts.items():
        setattr(o, key, val)
    it = np.zeros(k, dtype=np.int32)
    rel = np.zeros(k)
    st = np.zeros(k, dtype=np.int32)
    sms = np.zeros(k)
    pms = np.zeros(k)
    torch.cuda.synchronize()
    P = ctypes.POINTER
    status = lib.msdd_batch_run(k, meshes, coeffs, decs, ctypes.byref(s), ctypes.byref(o), bp, float(tol), int(maxit),
                                xp, int(nworkers), it.ctypes.data_as(P(ctypes.c_int)),
                                rel.ctypes.data_as(P(ctypes.c_double)), st.ctypes.data_as(P(ctypes.c_int)),
                                sms.ctypes.data_as(P(ctypes.c_double)), pms.ctypes.data_as(P(ctypes.c_double)))
    if not allow_fail:
        _check(status)
    return xs, it, rel, st, sms, pms


def fine_layout(n, parts, overlap, dirichlet_faces=0b1):
    """(P, 4) int array: Neumann-box node counts (nx, ny, nz) and row offset of each fine subdomain."""
    lib = load()
    mesh, d = make_mesh(n, dirichlet_faces), _decomp(parts, overlap)
    cnt = ctypes.c_int()
    _check(lib.msdd_fine_layout(ctypes.byref(mesh), ctypes.byref(d), None, 0, ctypes.byref(cnt)))
    out = np.zeros(4 * cnt.value, dtype=np.int32)
    _check(lib.msdd_fine_layout(ctypes.byref(mesh), ctypes.byref(d), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                out.size, ctypes.byref(cnt)))
    return out.reshape(-1, 4)


def nn_patches(n, kappa, parts, overlap, dirichlet_faces=0b1):
    """Network inputs (P, NN_IN) float32 CUDA of all fine subdomains (2D scalar kappa, CUDA float64)."""
    torch = _torch()
    lib = load()
    mesh, d = make_mesh(n, dirichlet_faces), _decomp(parts, overlap)
    kappa = kappa.to(device="cuda", dtype=torch.float64).contiguous()
    c = Coeff()
    c.kind = 0
    c.data = kappa.data_ptr()
    P = fine_layout(n, parts, overlap, dirichlet_faces).shape[0]
    X = torch.empty((P, NN_IN), dtype=torch.float32, device="cuda")
    _check(lib.msdd_nn_patches(ctypes.byref(mesh), ctypes.byref(c), ctypes.byref(d), ctypes.c_void_p(X.data_ptr()),
                               _stream()))
    return X


def nn_start_vectors(n, parts, overlap, Y, dirichlet_faces=0b1):
    """Grid vectors Y (P, NN_OUT) -> start vectors (rows of fine_layout, NN_NVEC) float64 CUDA."""
    torch = _torch()
    lib = load()
    mesh, d = make_mesh(n, dirichlet_faces), _decomp(parts, overlap)
    lay = fine_layout(n, parts, overlap, dirichlet_faces)
    rows = int(lay[-1, 3] + lay[-1, 0] * lay[-1, 1] * lay[-1, 2])
    Y = Y.to(device="cuda", dtype=torch.float32).contiguous()
    out = torch.empty((rows, NN_NVEC), dtype=torch.float64, device="cuda")
    _check(lib.msdd_nn_start_vectors(ctypes.byref(mesh), ctypes.byref(d), ctypes.c_void_p(Y.data_ptr()),
                                     ctypes.c_void_p(out.data_ptr()), _stream()))
    return out


class WarmStartNet:
    """Parameters (FP32 master copy) and Adam state of the warm-start network;
    forward, loss/gradient and Adam steps run in the library's kernels."""

    def __init__(self, params):
        torch = _torch()
        self._lib = load()
        self.params = params.to(device="cuda", dtype=torch.float32).contiguous().clone()
        assert self.params.numel() == NN_NPARAM
        self.m1 = torch.zeros_like(self.params)
        self.m2 = torch.zeros_like(self.params)
        self.t = 0
        self._work = None

    def _workspace(self, batch):
        torch = _torch()
        nbytes = self._lib.msdd_nn_workspace_bytes(int(batch))
        if self._work is None or self._work.numel() * 4 < nbytes:
            self._work = torch.empty((nbytes + 3) // 4, dtype=torch.float32, device="cuda")
        return self._work

    def forward(self, X):
        torch = _torch()
        X = X.to(device="cuda", dtype=torch.float32).contiguous()
        out = torch.empty((X.shape[0], NN_OUT), dtype=torch.float32, device="cuda")
        w = self._workspace(X.shape[0])
        _check(self._lib.msdd_nn_forward(ctypes.c_void_p(self.params.data_ptr()), int(X.shape[0]),
                                         ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                         ctypes.c_void_p(w.data_ptr()), _stream()))
        return out

    def loss_grad(self, X, T, m):
        """Batch loss (float64 0-d CUDA tensor) and gradient (NN_NPARAM float32)."""
        torch = _torch()
        X = X.to(device="cuda", dtype=torch.float32).contiguous()
        T = T.to(device="cuda", dtype=torch.float32).contiguous()
        m = m.to(device="cuda", dtype=torch.int32).contiguous()
        loss = torch.empty((), dtype=torch.float64, device="cuda")
        grad = torch.empty_like(self.params)
        w = self._workspace(X.shape[0])
        _check(self._lib.msdd_nn_loss_grad(ctypes.c_void_p(self.params.data_ptr()), int(X.shape[0]),
                                           ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(T.data_ptr()),
                                           ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                           ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(w.data_ptr()), _stream()))
        return loss, grad

    def adam_step(self, grad, lr):
        self.t += 1
        _check(self._lib.msdd_nn_adam(ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                      ctypes.c_void_p(self.m1.data_ptr()), ctypes.c_void_p(self.m2.data_ptr()),
                                      self.t, ctypes.c_float(lr), _stream()))
