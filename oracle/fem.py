"""Q1 conforming finite elements for -div(K grad u) = f on a box (oracle).

Test infrastructure only.  Follows Section 3.4 (Eq. ScalarBVP and the forms
a_h, a_tau, l that follow it): a_tau(u, v) = int_tau (K grad u) . grad v, and
a_h is the sum over elements.  The mesh is a structured grid of
nx x ny (x nz) equal boxes on [0, 1]^d; K is constant on each element.

Conventions shared with the CUDA library (they are interface facts, not code):
  * element (ex, ey, ez) has flat index ex + nx * (ey + ny * ez);
  * node (ix, iy, iz) has flat index ix + (nx+1) * (iy + (ny+1) * iz);
  * the local nodes of an element are ordered lexicographically, x fastest:
    local node a <-> offsets (a & 1, (a >> 1) & 1, (a >> 2) & 1);
  * Dirichlet faces are a bitmask: bit 2*d is the face x_d = 0, bit 2*d+1 the
    face x_d = 1; Dirichlet nodes are eliminated (u = 0 there);
  * unknowns are the remaining nodes, numbered lexicographically (x fastest)
    within the box of non-Dirichlet nodes;
  * a scalar coefficient is one value per element; a tensor coefficient is
    (kxx, kyy, kxy) per element in 2D and (kxx, kyy, kzz, kyz, kxz, kxy) in 3D.
"""
import itertools
import numpy as np
import scipy.sparse as sp


class Mesh:
    def __init__(self, n, dirichlet_faces=0b1):
        self.n = tuple(int(v) for v in n)
        self.dim = len(self.n)
        assert self.dim in (2, 3)
        self.h = tuple(1.0 / v for v in self.n)
        self.dirichlet_faces = int(dirichlet_faces)
        self.nodes_per_axis = tuple(v + 1 for v in self.n)
        self.num_nodes = int(np.prod(self.nodes_per_axis))
        self.num_elements = int(np.prod(self.n))
        lo, hi = [], []
        for d in range(self.dim):
            lo.append(1 if (self.dirichlet_faces >> (2 * d)) & 1 else 0)
            hi.append(self.n[d] - 1 if (self.dirichlet_faces >> (2 * d + 1)) & 1 else self.n[d])
        self.unknown_lo = tuple(lo)
        self.unknown_hi = tuple(hi)          # inclusive
        self.unknown_shape = tuple(h - l + 1 for l, h in zip(lo, hi))
        self.num_unknowns = int(np.prod(self.unknown_shape))

    # --- index helpers -------------------------------------------------
    def node_index(self, idx):
        """Flat node index of integer coordinates idx = (ix, iy[, iz])."""
        out = 0
        stride = 1
        for d in range(self.dim):
            out = out + np.asarray(idx[d]) * stride
            stride *= self.nodes_per_axis[d]
        return out

    def node_to_unknown(self):
        """Array over all nodes: unknown number, or -1 for Dirichlet nodes."""
        m = -np.ones(self.num_nodes, dtype=np.int64)
        grids = np.meshgrid(*[np.arange(l, h + 1) for l, h in zip(self.unknown_lo, self.unknown_hi)],
                            indexing="ij")
        # lexicographic, x fastest: unknown index = ux + sx * (uy + sy * uz)
        unk = np.zeros(grids[0].shape, dtype=np.int64)
        stride = 1
        for d in range(self.dim):
            unk = unk + (grids[d] - self.unknown_lo[d]) * stride
            stride *= self.unknown_shape[d]
        m[self.node_index(grids).ravel()] = unk.ravel()
        return m

    def element_nodes(self):
        """(num_elements, 2^d) flat node indices of each element, local order x fastest."""
        grids = np.meshgrid(*[np.arange(v) for v in self.n], indexing="ij")
        # flat element index e = ex + nx*(ey + ny*ez): build in that order
        e_idx = np.zeros(grids[0].shape, dtype=np.int64)
        stride = 1
        for d in range(self.dim):
            e_idx = e_idx + grids[d] * stride
            stride *= self.n[d]
        out = np.zeros((self.num_elements, 2 ** self.dim), dtype=np.int64)
        for a in range(2 ** self.dim):
            off = [(a >> d) & 1 for d in range(self.dim)]
            nodes = self.node_index([grids[d] + off[d] for d in range(self.dim)])
            out[e_idx.ravel(), a] = nodes.ravel()
        return out

    def element_coords(self):
        """(num_elements, d) integer lower-corner coordinates of each element."""
        out = np.zeros((self.num_elements, self.dim), dtype=np.int64)
        e = np.arange(self.num_elements)
        for d in range(self.dim):
            out[:, d] = e % self.n[d]
            e = e // self.n[d]
        return out


def tensor_from_coefficient(dim, coeff):
    """(num_elements, d, d) conductivity tensors from scalar or tensor input."""
    coeff = np.asarray(coeff, dtype=np.float64)
    if coeff.ndim == 1:
        return coeff[:, None, None] * np.eye(dim)[None]
    K = np.zeros((coeff.shape[0], dim, dim))
    if dim == 2:
        K[:, 0, 0], K[:, 1, 1] = coeff[:, 0], coeff[:, 1]
        K[:, 0, 1] = K[:, 1, 0] = coeff[:, 2]
    else:
        K[:, 0, 0], K[:, 1, 1], K[:, 2, 2] = coeff[:, 0], coeff[:, 1], coeff[:, 2]
        K[:, 1, 2] = K[:, 2, 1] = coeff[:, 3]
        K[:, 0, 2] = K[:, 2, 0] = coeff[:, 4]
        K[:, 0, 1] = K[:, 1, 0] = coeff[:, 5]
    return K


def q1_element_matrix_quadrature(h, K):
    """Element stiffness int_tau (K grad phi_b) . grad phi_a by 2^d-point Gauss.

    h: element edge lengths (d,), K: (d, d) constant tensor.  The Q1 basis on
    [0, h_1] x ... is the product of 1D hat functions; the integrand is a
    polynomial of degree <= 2 per variable, integrated exactly by 2-point
    Gauss-Legendre in each direction.
    """
    dim = len(h)
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    nloc = 2 ** dim
    A = np.zeros((nloc, nloc))
    vol = float(np.prod(h))
    for qp in itertools.product(range(2), repeat=dim):
        xi = [g[q] for q in qp]                    # reference coordinates in [0,1]
        grads = np.zeros((nloc, dim))
        for a in range(nloc):
            bits = [(a >> d) & 1 for d in range(dim)]
            # phi_a = prod_d (bits_d ? xi_d : 1 - xi_d)
            vals = [xi[d] if bits[d] else 1.0 - xi[d] for d in range(dim)]
            for d in range(dim):
                dv = (1.0 if bits[d] else -1.0) / h[d]
                prod = dv
                for e in range(dim):
                    if e != d:
                        prod *= vals[e]
                grads[a, d] = prod
        w = vol / nloc                              # Gauss weights 1/2 per axis
        A += w * grads @ K @ grads.T
    return A


def q1_element_matrix_2d_scalar(kappa, hx, hy):
    """Closed form of the 2D Q1 element stiffness for scalar kappa.

    Tensor-product structure: the bilinear basis is phi_i(x) psi_j(y), so
    int grad(phi psi) . grad(phi' psi') = (int phi' phi'') (int psi psi')
    + (int phi phi') (int psi' psi''), i.e. kron of 1D stiffness and mass
    matrices.  Local order x fastest: a = ax + 2 ay.
    """
    k1x = np.array([[1.0, -1.0], [-1.0, 1.0]]) / hx
    m1x = np.array([[2.0, 1.0], [1.0, 2.0]]) * hx / 6.0
    k1y = np.array([[1.0, -1.0], [-1.0, 1.0]]) / hy
    m1y = np.array([[2.0, 1.0], [1.0, 2.0]]) * hy / 6.0
    # index a = ax + 2 ay  ->  kron(y-part, x-part)
    return kappa * (np.kron(m1y, k1x) + np.kron(k1y, m1x))


def element_matrices(mesh, coeff):
    """(len(coeff), 2^d, 2^d) element stiffness matrices of the elements whose
    coefficients are given (all elements of the mesh, or a subset)."""
    K = tensor_from_coefficient(mesh.dim, coeff)
    coeff = np.asarray(coeff, dtype=np.float64)
    if coeff.ndim == 1:
        ref = q1_element_matrix_quadrature(mesh.h, np.eye(mesh.dim))
        return coeff[:, None, None] * ref[None]
    # general tensor: the element matrix is linear in K; build from the
    # d*(d+1)/2 basis tensors
    out = np.zeros((coeff.shape[0], 2 ** mesh.dim, 2 ** mesh.dim))
    for i in range(mesh.dim):
        for j in range(mesh.dim):
            E = np.zeros((mesh.dim, mesh.dim))
            E[i, j] = 1.0
            ref = q1_element_matrix_quadrature(mesh.h, E)
            out += K[:, i, j][:, None, None] * ref[None]
    return out


def assemble_neumann(mesh, coeff, element_mask=None):
    """All-node stiffness matrix sum_{tau in mask} a_tau (sparse, num_nodes^2)."""
    Ke = element_matrices(mesh, coeff)
    en = mesh.element_nodes()
    if element_mask is not None:
        Ke = Ke[element_mask]
        en = en[element_mask]
    nloc = en.shape[1]
    rows = np.repeat(en, nloc, axis=1).ravel()
    cols = np.tile(en, (1, nloc)).ravel()
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(mesh.num_nodes, mesh.num_nodes))


def assemble_system(mesh, coeff):
    """Global stiffness on the unknowns (Dirichlet nodes eliminated), CSR."""
    An = assemble_neumann(mesh, coeff)
    n2u = mesh.node_to_unknown()
    keep = np.nonzero(n2u >= 0)[0]            # ascending node index == ascending unknown
    return An[keep][:, keep].tocsr()


def load_vector(mesh, f=1.0):
    """l(v) = int f v for constant f (no Neumann flux), on the unknowns."""
    en = mesh.element_nodes()
    vol = float(np.prod(mesh.h))
    b = np.zeros(mesh.num_nodes)
    np.add.at(b, en.ravel(), f * vol / en.shape[1])
    return b[mesh.node_to_unknown() >= 0]
