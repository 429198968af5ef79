"""Method mode of the CPU oracle: the same multilevel method with the fine
level computed the way the method is run at scale (test infrastructure only).

The dense oracle (method.py) solves every fine GEVP completely by Jacobi on
the spectrally transformed pencil, which costs minutes per subdomain at the
sizes of the 2D 512 x 512 workload.  Method mode keeps everything else of the
dense oracle (decomposition, partition of unity, coarse generating-system
GEVPs of Section 4.2, Galerkin matrices, the additive preconditioner and CG)
and replaces, on the fine level only:

  * the dense Cholesky factors of the Dirichlet matrices A_i by band
    Cholesky factors (Section 4.3: a direct solver per subdomain);
  * the complete eigendecomposition by block subspace iteration with
    Rayleigh-Ritz on the shift-inverted pencil (Section 4.2 uses ARPACK's
    shift-invert mode): Y = (Abar_i + sigma B_i)^{-1} B_i X, then the
    projected pencil (Y^T Abar Y, Y^T B Y) is solved exactly and X = Y Q.
    Iteration stops when the m = min(nev_max, #{theta < eta}) selected pairs
    have relative residuals |Abar x - theta B x| / |B x| below `tol` and,
    when m < nev_max, the next Ritz value, which decides the selection, is
    settled: its residual times max(1, theta) is below a tenth of its
    distance to eta.  (Past eta the spectrum often holds a large cluster at
    lambda = 1 from functions where chi = 1, which a block of nev_max + 8
    vectors resolves only slowly.)

Plain FP64; band routines in linalg.c; products through numpy/scipy sparse.
Readings: sigma = 1e-2 (the paper leaves the shift open), block size
nev_max + 8, a seeded Gaussian start block per subdomain.
"""
import numpy as np
import scipy.sparse as sp

from . import fem
from . import linalg
from . import method
from .decomposition import Decomposition


def local_neumann(Ke, en, element_mask, nn, num_nodes):
    """Abar_i (Eq. locala_cg) as a sparse matrix over the Neumann nodes nn of
    one subdomain: the element matrices of its elements, Dirichlet nodes
    dropped."""
    pos = -np.ones(num_nodes, dtype=np.int64)
    pos[nn] = np.arange(len(nn))
    loc = pos[en[element_mask]]
    nloc = loc.shape[1]
    rows = np.repeat(loc, nloc, axis=1).ravel()
    cols = np.tile(loc, (1, nloc)).ravel()
    vals = Ke[element_mask].ravel()
    keep = (rows >= 0) & (cols >= 0)
    n = len(nn)
    return sp.csr_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n))


def rayleigh_ritz(H, M):
    """Ritz pairs of the projected pencil H c = theta M c: M = V diag(s) V^T
    (Jacobi), directions with s <= 1e-14 max(s) dropped, then Jacobi on
    T^T H T with T = V diag(s^{-1/2}).  Returns ascending theta and Q with
    Q^T M Q = I."""
    s, V = linalg.jacobi_eigh(M)
    keep = s > 1e-14 * max(s.max(), 0.0)
    T = V[:, keep] / np.sqrt(s[keep])[None, :]
    theta, U = linalg.jacobi_eigh(T.T @ H @ T)
    return theta, T @ U


def subspace_iteration(Abar, B, KL, nev_max, eta, p, tol, maxit, rng):
    """Lowest eigenpairs of Abar w = lambda B w by block subspace iteration
    with the band factor KL of Abar + sigma B.  Returns (theta, X, iterations)
    with X^T B X = I and theta ascending (p Ritz pairs)."""
    n = Abar.shape[0]
    p = min(p, n)
    X = rng.standard_normal((n, p))
    theta = np.zeros(0)
    for it in range(1, maxit + 1):
        Y = linalg.band_solve(KL, B @ X)
        theta, Q = rayleigh_ritz(Y.T @ (Abar @ Y), Y.T @ (B @ Y))
        X = Y @ Q
        if X.shape[1] < p:                       # refill directions lost to rank deficiency
            X = np.concatenate([X, rng.standard_normal((n, p - X.shape[1]))], axis=1)
            continue
        BX = B @ X
        R = Abar @ X - BX * theta[None, :]
        res = np.linalg.norm(R, axis=0) / np.maximum(np.linalg.norm(BX, axis=0), 1e-300)
        m = method.select_count(theta, nev_max, eta)
        done = bool(np.all(res[:m] <= tol))
        if done and m < min(nev_max, p):
            # the next Ritz value decides the selection: it must be settled
            # clear of eta (error estimate below a tenth of its distance)
            done = res[m] * max(1.0, abs(theta[m])) <= 0.1 * abs(theta[m] - eta)
        if done:
            return theta, X, it
    return theta, X, -maxit


# ---- fine-level work, one subdomain per task (also run in spawned worker
# processes, which rebuild the inputs once from the problem description)
_W = {}


def _worker_init(n, dirichlet_faces, coeff, parts, overlap, levels, group, opts):
    mesh = fem.Mesh(n, dirichlet_faces)
    dec = Decomposition(mesh, parts, overlap, levels, group)
    chis, counts = dec.partition_of_unity()
    _W.update(mesh=mesh, dec=dec, chis=chis, counts=counts, Ke=fem.element_matrices(mesh, coeff),
              en=mesh.element_nodes(), A=fem.assemble_system(mesh, coeff).tocsr(),
              n2u=mesh.node_to_unknown(), opts=opts)


def _fine_local(i):
    """Fine subdomain i: Abar_i, B_i = X Abar_i X (b^1, Eq. cg_rhs_blf), the
    band factor of Abar_i + sigma B_i, subspace iteration, selection, and the
    band factor of the Dirichlet matrix A_i."""
    mesh, dec, o = _W["mesh"], _W["dec"], _W["opts"]
    s = dec.fine[i]
    nn = s.neumann_nodes()
    chi = _W["chis"][i]
    Abar = local_neumann(_W["Ke"], _W["en"], s.element_mask, nn, mesh.num_nodes)
    X = sp.diags(chi)
    B = (X @ Abar @ X).tocsr()
    K = (Abar + o["sigma"] * B).tocsr()
    KL = linalg.band_cholesky(linalg.to_band(K, linalg.half_bandwidth(K)))
    rng = np.random.default_rng([o["seed"], i])
    theta, Xr, its = subspace_iteration(Abar, B, KL, o["nev_max"], o["eta"], o["nev_max"] + o["extra"],
                                        o["tol"], o["maxit"], rng)
    m = method.select_count(theta, o["nev_max"], o["eta"])
    Wm = method.normalise_sign(Xr[:, :m])
    dn = s.dirichlet_nodes()
    du = _W["n2u"][dn]
    Ai = _W["A"][du][:, du]
    Li = linalg.band_cholesky(linalg.to_band(Ai, linalg.half_bandwidth(Ai)))
    keep = o["keep_local"]
    return dict(nn=nn, chi=chi, chi_dir=1.0 / _W["counts"][dn],
                Abar=Abar.toarray() if keep else None, B=B.toarray() if keep else None,
                lam=theta, m=m, W=Wm, dof=du, Ai=Ai.toarray() if keep else None, Li=Li,
                eig_iterations=its)


class MethodModeHierarchy(method.Hierarchy):
    """method.Hierarchy with band factors and subspace iteration on the fine
    level.  processes > 1 runs the fine subdomains in that many spawned
    worker processes (start it before any GPU use in the same process, or
    from a fresh interpreter)."""

    def __init__(self, mesh, coeff, parts, overlap, levels, group, nev_max, eta, sigma=1e-2, tol=1e-8,
                 extra=8, maxit=400, seed=0, keep_local=False, processes=1):
        self.opts = dict(sigma=sigma, tol=tol, extra=extra, maxit=maxit, seed=seed, nev_max=nev_max,
                         eta=eta, keep_local=keep_local)
        self.processes = processes
        self._args = (tuple(mesh.n), mesh.dirichlet_faces, np.asarray(coeff), tuple(parts), overlap, levels,
                      tuple(group))
        super().__init__(mesh, coeff, parts, overlap, levels, group, nev_max, eta, keep_local=keep_local)

    def _build_fine(self, keep_local):
        P = self.dec.num_subdomains(self.L)
        self.pou_counts = self.dec.partition_of_unity()[1]
        if self.processes > 1:
            import multiprocessing as mp
            from concurrent.futures import ProcessPoolExecutor
            with ProcessPoolExecutor(self.processes, mp_context=mp.get_context("spawn"),
                                     initializer=_worker_init, initargs=self._args + (self.opts,)) as ex:
                subs = list(ex.map(_fine_local, range(P), chunksize=max(1, P // (4 * self.processes))))
        else:
            _worker_init(*self._args, self.opts)
            subs = [_fine_local(i) for i in range(P)]
            _W.clear()
        lev = method.Level()
        lev.subs = subs
        rows, cols, vals = [], [], []
        col = 0
        lev.col_range = []
        for s in subs:
            u = self.n2u[s["nn"]]
            for k in range(s["m"]):
                phi = s["chi"] * s["W"][:, k]
                nz = phi != 0.0
                rows.append(u[nz]); cols.append(np.full(nz.sum(), col)); vals.append(phi[nz])
                col += 1
            lev.col_range.append((col - s["m"], col))
        lev.P_coarse = sp.csc_matrix((np.concatenate(vals) if vals else np.zeros(0),
                                      (np.concatenate(rows) if rows else np.zeros(0, int),
                                       np.concatenate(cols) if cols else np.zeros(0, int))),
                                     shape=(self.n, col))
        lev.P = None
        self.levels[self.L] = lev

    def _fine_solve(self, s, r):
        return linalg.band_solve(s["Li"], r)


# ---- a bounded sample of the fine level (for workloads too large for a
# full oracle run on the host): workers build only what the sampled
# subdomains need (their element matrices, the partition of unity)
def _sample_init(n, dirichlet_faces, coeff, parts, overlap, levels, group, opts):
    mesh = fem.Mesh(n, dirichlet_faces)
    dec = Decomposition(mesh, parts, overlap, levels, group)
    chis, counts = dec.partition_of_unity()
    _W.update(mesh=mesh, dec=dec, chis=chis, coeff=np.asarray(coeff), en=mesh.element_nodes(), opts=opts)


def _sample_local(i):
    mesh, dec, o = _W["mesh"], _W["dec"], _W["opts"]
    s = dec.fine[i]
    nn = s.neumann_nodes()
    chi = _W["chis"][i]
    mask = s.element_mask
    Ke = fem.element_matrices(mesh, _W["coeff"][mask])
    idx = np.nonzero(mask)[0]
    full_mask = np.ones(len(idx), dtype=bool)
    Abar = local_neumann(Ke, _W["en"][idx], full_mask, nn, mesh.num_nodes)
    X = sp.diags(chi)
    B = (X @ Abar @ X).tocsr()
    K = (Abar + o["sigma"] * B).tocsr()
    KL = linalg.band_cholesky(linalg.to_band(K, linalg.half_bandwidth(K)))
    rng = np.random.default_rng([o["seed"], i])
    theta, Xr, its = subspace_iteration(Abar, B, KL, o["nev_max"], o["eta"], o["nev_max"] + o["extra"], o["tol"],
                                        o["maxit"], rng)
    return dict(lam=theta, m=method.select_count(theta, o["nev_max"], o["eta"]), eig_iterations=its)


def fine_level_sample(n, dirichlet_faces, coeff, parts, overlap, levels, group, nev_max, eta, sample, processes,
                      sigma=1e-2, tol=1e-8, extra=8, maxit=400, seed=0):
    """Method-mode fine-level eigenpairs (Ritz values, selected counts) of the
    fine subdomains listed in `sample`, in `processes` spawned workers."""
    opts = dict(sigma=sigma, tol=tol, extra=extra, maxit=maxit, seed=seed, nev_max=nev_max, eta=eta)
    args = (tuple(n), dirichlet_faces, np.asarray(coeff), tuple(parts), overlap, levels, tuple(group), opts)
    if processes > 1:
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        with ProcessPoolExecutor(min(processes, len(sample)), mp_context=mp.get_context("spawn"),
                                 initializer=_sample_init, initargs=args) as ex:
            return list(ex.map(_sample_local, sample))
    _sample_init(*args)
    out = [_sample_local(i) for i in sample]
    _W.clear()
    return out
