"""Multilevel spectral domain decomposition, plain FP64 CPU oracle.

Test infrastructure only: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it; the CUDA library never does.

Steps, in the paper's order and notation:
  1. Local Neumann forms abar_{l,i}(u, v) = sum_{tau in T_{h,l,i}} a_tau(u, v)
     (Eq. locala_cg) and the partition-of-unity weighted form
     b^1_{l,i}(u, v) = abar_{l,i}(chi u, chi v) (Eq. cg_rhs_blf, first line).
  2. Local GEVPs abar(w, v) = lambda b(w, v) (Eq. theGEVP), solved exactly:
     the spectral transformation b(p, v) = mu (a + b)(p, v), mu = 1/(1+lambda)
     (proof of the non-defectiveness lemma, Section 3.3) turns the pencil into
     a standard symmetric problem that the Jacobi method solves completely.
     On coarse levels only a generating system is available and
     ker A cap ker B is not trivial (Section 3.3 remark); the generators
     that the regularised LDL^T of Section 4.2 (Eq. evp_reg) finds dependent
     are dropped first (gevp_regularised).
  3. Coarse space V_{h,l-1} = span{ e chi w : lambda < eta } (Eq.
     coarse_space_def), at most nev_max per subdomain (Section 5.1.1 offers a
     fixed count or a threshold; both are applied, the smaller wins).
  4. Coarse levels built from the generating system of Section 4.2: own
     children's basis functions plus the restrictions of the neighbouring
     children's basis functions to Omega_{l,i}; chi_{l,i} keeps the own part.
  5. Dirichlet subspaces V_{h,l,i} (Eq. dirichlet_space) and the additive
     preconditioner B = sum_i R_i^T A_i^{-1} R_i over all levels plus the
     coarsest solve (Section 2.1, Eq. mlsdd), used in CG, stopped when
     ||b - A x^m|| < tol ||b - A x^0|| (Section 5) with x^0 = 0 and the
     Euclidean norm.

Readings where the paper is silent (listed with the others in the design
notes): on coarse levels the regularised LDL^T factors K = A + sigma B
(sigma = 1e-2) in generator order, and a pivot d_k <= tau K_kk is a null
pivot (tau = 1e-10 in 2D; 1e-6 in 3D, where it also drops generators that
are only nearly dependent; eps^{-1} -> 0); for the b^2 and b^3
forms on the fine level the common kernel is dropped by a rank threshold
1e-12 * max eigenvalue of (A + B); eigenvalues with mu <= 1e-13 are treated
as +infinity; an eigenvector is normalised to b(w, w) = 1 and signed so that
its entry of largest magnitude is positive; selection uses lambda < eta
strictly.
"""
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import scipy.sparse as sp

from . import fem
from . import linalg
from .decomposition import Decomposition

TOL_RANK = 1e-12
MU_INF = 1e-13


def _pool_size():
    return max(1, min(32, os.cpu_count() or 1))


def gevp(Abar, B, rank_reveal):
    """All eigenpairs of Abar w = lambda B w with finite lambda, ascending.

    Returns (lam, W) with W[:, k] b-orthonormal (W^T B W = I) and lam sorted
    ascending.  If rank_reveal, the common kernel of Abar and B is removed
    first (eigenvectors of Abar + B with eigenvalue <= TOL_RANK * max).
    """
    n = Abar.shape[0]
    S = Abar + B
    if rank_reveal:
        s, U = linalg.jacobi_eigh(S)
        keep = s > TOL_RANK * max(s.max(), 0.0)
        U = U[:, keep]
    else:
        U = np.eye(n)
    Ar = U.T @ Abar @ U
    Br = U.T @ B @ U
    Lc = linalg.cholesky(0.5 * ((Ar + Br) + (Ar + Br).T))
    # C = L^{-1} Br L^{-T}
    T = linalg.forward(Lc, Br)              # L^{-1} Br
    C = linalg.forward(Lc, T.T)             # L^{-1} (L^{-1} Br)^T = L^{-1} Br L^{-T}
    mu, V = linalg.jacobi_eigh(C)           # ascending mu
    order = np.argsort(-mu, kind="stable")  # descending mu == ascending lambda
    mu, V = mu[order], V[:, order]
    finite = mu > MU_INF
    mu, V = mu[finite], V[:, finite]
    W = U @ linalg.backward(Lc, V)          # w = U L^{-T} v
    W = W / np.sqrt(mu)[None, :]            # b(w, w) = v^T C v / mu = 1
    lam = 1.0 / mu - 1.0
    return lam, W


def gevp_regularised(Abar, B, sigma, tau):
    """All finite eigenpairs of the generating-system pencil of a coarse
    level (Section 4.2, Eq. evp_reg), ascending.

    The paper factors the pencil's matrix as L D L^T and replaces the zero
    pivots by 0 < eps << 1; the vectors that pass through the regularised
    pivots then have eigenvalues near eps (lambda ~ 0, kernel directions)
    or belong to ker B (lambda = infinity).  Reading, in the limit
    eps^{-1} -> 0 and with the shift of the spectral transformation: the
    matrix factored is K = Abar + sigma B, in generator order, and a pivot
    d_k <= tau K_kk is a null pivot, which drops generator k as dependent on
    the earlier ones in K-energy.  The pencil is then solved completely on
    the kept directions V = L^{-T}[:, kept] (span of the generating system
    less those dependencies) by gevp().  Returns (lam, W), W = V W_r with
    W^T B W = I, and the number of null pivots."""
    K = Abar + sigma * B
    L, d, null = linalg.ldlt_null(K, tau)
    keep = ~null
    n = Abar.shape[0]
    E = np.eye(n)[:, keep]
    V = linalg.backward(L, E)                  # L^T V = E: V = L^{-T} E (L unit lower)
    Ar = V.T @ Abar @ V
    Br = V.T @ B @ V
    lam, Wr = gevp(0.5 * (Ar + Ar.T), 0.5 * (Br + Br.T), rank_reveal=False)
    return lam, V @ Wr, int(null.sum())


def normalise_sign(W):
    """Flip each column so that its entry of largest magnitude is positive.

    Parity unpinned: a sign convention, not part of the method; no comparison
    with the CUDA path depends on it (spans and Ritz values are compared)."""
    W = W.copy()
    for k in range(W.shape[1]):
        i = int(np.argmax(np.abs(W[:, k])))
        if W[i, k] < 0:
            W[:, k] = -W[:, k]
    return W


def select_count(lam, nev_max, eta):
    """m = min(nev_max, #{lambda < eta}) (Eq. coarse_space_def, Section 5.1.1)."""
    return int(min(nev_max, int(np.sum(lam < eta))))


def fine_pencil(mesh, Ke, en, sub, chi, Ke_of_subdomain=False, blf=1, overlap_elements=None):
    """Dense Neumann matrix Abar_i (Eq. locala_cg: the element forms of
    T_{h,L,i} on all non-Dirichlet nodes of the closed subdomain) and the
    right-hand side B_i of one fine subdomain's GEVP, rows in its
    lexicographic Neumann-node order (Section 3.4, Eq. cg_rhs_blf):
      blf = 1: b^1(u, v) = abar(chi u, chi v),       B = X Abar X;
      blf = 2: b^2(u, v) = a_ring(chi u, chi v),     B = X Aring X, Aring the
               element forms of the subdomain's elements that also belong to
               another subdomain (overlap_elements[e], Eq. original_geneo);
      blf = 3: b^3(u, v) = abar(u - chi u, v - chi v), B = (I - X) Abar (I - X).
    en are the element nodes of the whole mesh, Ke the element matrices of
    the whole mesh (or, with Ke_of_subdomain, of the subdomain's elements in
    ascending order), chi the subdomain's partition of unity on its Neumann
    nodes (Section 2.3), X = diag(chi)."""
    nn = sub.neumann_nodes()
    pos = -np.ones(mesh.num_nodes, dtype=np.int64)
    pos[nn] = np.arange(len(nn))
    Abar = np.zeros((len(nn), len(nn)))
    Aring = np.zeros((len(nn), len(nn))) if blf == 2 else None
    for k, e in enumerate(np.nonzero(sub.element_mask)[0]):
        loc = pos[en[e]]
        ok = loc >= 0
        li = loc[ok]
        ke = (Ke[k] if Ke_of_subdomain else Ke[e])[np.ix_(ok, ok)]
        Abar[np.ix_(li, li)] += ke
        if blf == 2 and overlap_elements[e]:
            Aring[np.ix_(li, li)] += ke
    if blf == 1:
        B = chi[:, None] * Abar * chi[None, :]
    elif blf == 2:
        B = chi[:, None] * Aring * chi[None, :]
    elif blf == 3:
        w = 1.0 - chi
        B = w[:, None] * Abar * w[None, :]
    else:
        raise ValueError("blf must be 1, 2 or 3")
    return nn, Abar, B


def overlap_elements(dec):
    """Elements of the fine level that belong to at least two fine subdomains
    (the union over i of the element sets of Eq. original_geneo)."""
    cover = np.zeros_like(dec.fine[0].element_mask, dtype=np.int64)
    for s in dec.fine:
        cover += s.element_mask
    return cover >= 2


class Level:
    pass


class Hierarchy:
    """Result of the oracle set-up: all levels, spaces and factors."""

    def __init__(self, mesh, coeff, parts, overlap, levels, group, nev_max, eta,
                 keep_local=False, blf=1, sigma=1e-2, reg_tol=None):
        self.mesh = mesh
        self.nev_max = nev_max
        self.eta = eta
        self.blf = blf
        # coarse-level generating systems (Section 4.2): shift and null-pivot
        # threshold of the regularised LDL^T (readings; 1e-10 in 2D, 1e-6 in 3D)
        self.sigma = sigma
        self.reg_tol = reg_tol if reg_tol is not None else (1e-10 if mesh.dim == 2 else 1e-6)
        self.A = fem.assemble_system(mesh, coeff)
        self.n = self.A.shape[0]
        self.dec = Decomposition(mesh, parts, overlap, levels, group)
        self.L = self.dec.L
        self.n2u = mesh.node_to_unknown()
        self._coeff = coeff
        self.levels = {}
        self._build_fine(keep_local)
        for l in range(self.L - 1, 0, -1):
            self._build_coarse(l, keep_local)
        P0 = self.levels[1].P_coarse
        self.A0 = (P0.T @ (self.A @ P0))
        self.A0 = np.asarray(self.A0.todense() if sp.issparse(self.A0) else self.A0)
        self.A0 = 0.5 * (self.A0 + self.A0.T)
        self.n0 = self.A0.shape[0]
        self.L0 = linalg.cholesky(self.A0) if self.n0 > 0 else None

    # --- fine level -----------------------------------------------------
    def _build_fine(self, keep_local):
        mesh, dec = self.mesh, self.dec
        chis, counts = dec.partition_of_unity()
        self.pou_counts = counts
        Ke = fem.element_matrices(mesh, self._coeff)
        en = mesh.element_nodes()
        ovl = overlap_elements(dec) if self.blf == 2 else None

        def local(i):
            s = dec.fine[i]
            nn, Abar, B = fine_pencil(mesh, Ke, en, s, chis[i], blf=self.blf, overlap_elements=ovl)
            chi = chis[i]
            # b^2 and b^3 have larger kernels than b^1: take the rank-revealing
            # route (complement of ker Abar cap ker B) for them
            lam, W = gevp(Abar, B, rank_reveal=self.blf != 1)
            m = select_count(lam, self.nev_max, self.eta)
            Wm = normalise_sign(W[:, :m])
            dn = s.dirichlet_nodes()
            du = self.n2u[dn]
            chi_dir = 1.0 / counts[dn]          # chi_i on the Dirichlet-space nodes (Section 2.3)
            Ai = np.asarray(self.A[du][:, du].todense())
            Li = linalg.cholesky(Ai)
            return dict(nn=nn, chi=chi, chi_dir=chi_dir, Abar=Abar if keep_local else None,
                        B=B if keep_local else None, lam=lam, m=m, W=Wm,
                        dof=du, Ai=Ai if keep_local else None, Li=Li)

        P = self.dec.num_subdomains(self.L)
        with ThreadPoolExecutor(_pool_size()) as ex:
            subs = list(ex.map(local, range(P)))
        lev = Level()
        lev.subs = subs
        # fine basis functions phi = e chi w in unknown coordinates
        rows, cols, vals = [], [], []
        col = 0
        lev.col_range = []
        for i, s in enumerate(subs):
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
        lev.P = None          # P_L = identity
        self.levels[self.L] = lev

    # --- coarse levels ----------------------------------------------------
    def _build_coarse(self, l, keep_local):
        """Level l (0 < l < L): GEVPs on generating systems, Section 4.2."""
        mesh, dec = self.mesh, self.dec
        child = self.levels[l + 1]
        Pl = child.P_coarse                     # n x n_l basis of V_{h,l} in fine coords
        Pl_dense_cols = Pl.tocsc()
        Al = np.asarray((Pl.T @ (self.A @ Pl)).todense())
        Al = 0.5 * (Al + Al.T)
        keep = self.n2u >= 0
        unk_nodes = np.nonzero(keep)[0]

        def local(i):
            own = dec.members[l][i]
            nbr = dec.neighbours(l, i)
            own_cols = np.concatenate([np.arange(*child.col_range[j]) for j in own]) if own else np.zeros(0, int)
            nbr_cols = np.concatenate([np.arange(*child.col_range[j]) for j in nbr]) if nbr else np.zeros(0, int)
            gen = np.concatenate([own_cols, nbr_cols]).astype(np.int64)
            G = Pl_dense_cols[:, gen]
            An = fem.assemble_neumann(mesh, self._coeff, dec.element_mask[l][i])
            An = An[unk_nodes][:, unk_nodes]
            Abar = np.asarray((G.T @ (An @ G)).todense())
            Abar = 0.5 * (Abar + Abar.T)
            x = np.concatenate([np.ones(len(own_cols)), np.zeros(len(nbr_cols))])
            B = x[:, None] * Abar * x[None, :]
            lam, W, nnull = gevp_regularised(Abar, B, self.sigma, self.reg_tol)
            m = select_count(lam, self.nev_max, self.eta)
            Wm = normalise_sign(W[:, :m])
            Ai = Al[np.ix_(own_cols, own_cols)]
            Li = linalg.cholesky(Ai) if len(own_cols) else None
            return dict(own=own, nbr=nbr, own_cols=own_cols, gen=gen, null_pivots=nnull,
                        Abar=Abar if keep_local else None, B=B if keep_local else None,
                        lam=lam, m=m, W=Wm, Ai=Ai if keep_local else None, Li=Li)

        P = dec.num_subdomains(l)
        with ThreadPoolExecutor(_pool_size()) as ex:
            subs = list(ex.map(local, range(P)))
        lev = Level()
        lev.subs = subs
        lev.P = Pl                                # V_{h,l} basis, fine coordinates
        lev.A_level = Al
        # next coarse basis: phi = e chi w = sum over own generators only
        blocks, col = [], 0
        lev.col_range = []
        Z = np.zeros((Pl.shape[1], 0))
        zcols = []
        for s in subs:
            nown = len(s["own_cols"])
            for k in range(s["m"]):
                z = np.zeros(Pl.shape[1])
                z[s["own_cols"]] = s["W"][:nown, k]
                zcols.append(z)
            lev.col_range.append((col, col + s["m"]))
            col += s["m"]
        lev.Z = np.stack(zcols, axis=1) if zcols else np.zeros((Pl.shape[1], 0))
        lev.P_coarse = sp.csc_matrix(Pl @ sp.csc_matrix(lev.Z))
        self.levels[l] = lev

    # --- preconditioner and CG --------------------------------------------
    def _fine_solve(self, s, r):
        """A_i^{-1} r for fine subdomain s (Eq. dirichlet_space), from its factor."""
        return linalg.cho_solve(s["Li"], r)

    def _fine_local_solves(self, r):
        """[A_i^{-1} R_i r for every fine subdomain i], in subdomain order."""
        return [self._fine_solve(s, r[s["dof"]]) for s in self.levels[self.L].subs]

    def _fine_sum(self, r, restricted=False):
        """sum_i R_i^T A_i^{-1} R_i r over the fine subdomains (restricted:
        each local solution weighted by chi_i first)."""
        z = np.zeros_like(r)
        for s, y in zip(self.levels[self.L].subs, self._fine_local_solves(r)):
            z[s["dof"]] += s["chi_dir"] * y if restricted else y
        return z

    def apply_preconditioner(self, r):
        """z = B r, the additive multilevel Schwarz preconditioner."""
        z = self._fine_sum(r)
        for l in range(self.L - 1, 0, -1):
            lev = self.levels[l]
            rl = lev.P.T @ r
            zl = np.zeros_like(rl)
            for s in lev.subs:
                if s["Li"] is not None:
                    zl[s["own_cols"]] += linalg.cho_solve(s["Li"], rl[s["own_cols"]])
            z += lev.P @ zl
        P0 = self.levels[1].P_coarse
        if self.n0 > 0:
            z += P0 @ linalg.cho_solve(self.L0, P0.T @ r)
        return z

    def apply_level(self, l, r, restricted=False):
        """z = B_l r, the part of the additive preconditioner on level l alone:
        l = L the fine local solves (restricted: prolongation weighted by chi_i,
        restricted additive Schwarz), 0 < l < L the solves on the own
        generators of level l, l = 0 the coarsest solve (Section 2.1,
        Eq. mlsdd).  The additive preconditioner is the sum over l."""
        z = np.zeros_like(r)
        if l == self.L:
            z = self._fine_sum(r, restricted)
        elif l > 0:
            lev = self.levels[l]
            rl = lev.P.T @ r
            zl = np.zeros_like(rl)
            for s in lev.subs:
                if s["Li"] is not None:
                    zl[s["own_cols"]] += linalg.cho_solve(s["Li"], rl[s["own_cols"]])
            z = lev.P @ zl
        elif self.n0 > 0:
            P0 = self.levels[1].P_coarse
            z = P0 @ linalg.cho_solve(self.L0, P0.T @ r)
        return z

    def apply_hybrid(self, r):
        """z = B_h r, the hybrid form used with GMRES in Section 5 (Tabs. 4-6):
        multiplicative subspace correction over the levels, restricted
        additive Schwarz within the fine level (Section 2.1, Eq.
        subspace_iteration applied level after level).  Reading: one sweep
        from the fine level to the coarsest, z <- z + B_l (r - A z); on the
        coarse levels the own-generator spaces do not overlap, so restricted
        and plain additive Schwarz coincide there."""
        z = self.apply_level(self.L, r, restricted=True)
        for l in range(self.L - 1, -1, -1):
            z = z + self.apply_level(l, r - self.A @ z)
        return z

    def apply_one_level(self, r):
        """z = sum_i R_i^T A_i^{-1} R_i r over the fine subdomains only (no coarse space)."""
        return self._fine_sum(r)

    def coarse_dims(self):
        """n_l for l = L-1 ... 0: dimension of each coarse space."""
        out = {}
        for l in range(self.L, 0, -1):
            out[l - 1] = self.levels[l].P_coarse.shape[1]
        return out

    def eigenvalues(self, l):
        return [s["lam"] for s in self.levels[l].subs]

    def counts(self, l):
        return [s["m"] for s in self.levels[l].subs]


def gmres(A, b, precond, tol=1e-8, restart=200, maxit=1000, flexible=False):
    """Right-preconditioned GMRES(restart) with modified Gram-Schmidt Arnoldi
    and Givens rotations (Saad and Schultz): x = M y minimises ||b - A M y||
    over the Krylov space of A M; x0 = 0; the run stops when the residual
    estimate of the Arnoldi process falls below tol * ||b|| (Section 5's
    stopping rule on the solver's own residual, as the recursive residual
    for CG) or the true residual at the end of a cycle does; a cycle that
    ends at the restart length restarts from the true residual.
    flexible=True is Saad's flexible GMRES: the
    preconditioned vectors z_k = M v_k are kept and the cycle's update is
    Z y, which minimises ||r - A Z y|| even when M changes from step to step
    (in exact arithmetic the same iterates as the plain form for a fixed M).
    Returns (x, iterations, history of ||r||/||b||)."""
    n = b.shape[0]
    x = np.zeros_like(b)
    bn = np.linalg.norm(b)
    hist = [1.0]
    if bn == 0.0:
        return x, 0, hist
    it = 0
    r = b.copy()
    while it < maxit:
        beta = np.linalg.norm(r)
        V = np.zeros((n, restart + 1))
        H = np.zeros((restart + 1, restart))
        cs, sn = np.zeros(restart), np.zeros(restart)
        g = np.zeros(restart + 1)
        g[0] = beta
        V[:, 0] = r / beta
        Z = np.zeros((n, restart)) if flexible else None
        k = 0
        for k in range(restart):
            z = precond(V[:, k])
            if flexible:
                Z[:, k] = z
            w = A @ z
            for i in range(k + 1):
                H[i, k] = V[:, i] @ w
                w = w - H[i, k] * V[:, i]
            H[k + 1, k] = np.linalg.norm(w)
            if H[k + 1, k] > 0.0:
                V[:, k + 1] = w / H[k + 1, k]
            for i in range(k):                      # previous rotations on the new column
                t = cs[i] * H[i, k] + sn[i] * H[i + 1, k]
                H[i + 1, k] = -sn[i] * H[i, k] + cs[i] * H[i + 1, k]
                H[i, k] = t
            den = np.hypot(H[k, k], H[k + 1, k])
            cs[k], sn[k] = H[k, k] / den, H[k + 1, k] / den
            H[k, k] = den
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            it += 1
            hist.append(abs(g[k + 1]) / bn)
            if abs(g[k + 1]) < tol * bn or it >= maxit:
                break
        y = np.linalg.solve(np.triu(H[:k + 1, :k + 1]), g[:k + 1])
        x = x + (Z[:, :k + 1] @ y if flexible else precond(V[:, :k + 1] @ y))
        r = b - A @ x
        if abs(g[k + 1]) < tol * bn or np.linalg.norm(r) < tol * bn or it >= maxit:
            break
    return x, it, hist


def pcg(A, b, precond, tol=1e-8, maxit=1000, x0=None):
    """Preconditioned CG; stops when ||r_m||_2 < tol * ||r_0||_2.

    Returns (x, iterations, history of ||r||/||r_0||, alphas, betas).
    """
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b - A @ x
    r0 = np.linalg.norm(r)
    hist = [1.0]
    alphas, betas = [], []
    if r0 == 0.0:
        return x, 0, hist, alphas, betas
    z = precond(r)
    p = z.copy()
    rz = r @ z
    it = 0
    while it < maxit:
        q = A @ p
        alpha = rz / (p @ q)
        x += alpha * p
        r -= alpha * q
        it += 1
        alphas.append(alpha)
        rel = np.linalg.norm(r) / r0
        hist.append(rel)
        if rel < tol:
            break
        z = precond(r)
        rz_new = r @ z
        beta = rz_new / rz
        betas.append(beta)
        rz = rz_new
        p = z + beta * p
    return x, it, hist, alphas, betas


def lanczos_condition(alphas, betas):
    """Extreme eigenvalues of the CG Lanczos tridiagonal (estimate of kappa(BA))."""
    k = len(alphas)
    if k == 0:
        return 1.0, 1.0
    T = np.zeros((k, k))
    for j in range(k):
        T[j, j] = 1.0 / alphas[j] + (betas[j - 1] / alphas[j - 1] if j > 0 else 0.0)
        if j + 1 < k and j < len(betas):
            T[j, j + 1] = T[j + 1, j] = np.sqrt(betas[j]) / alphas[j]
    w, _ = linalg.jacobi_eigh(T)
    return w[0], w[-1]
