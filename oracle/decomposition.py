"""Hierarchical box domain decomposition and partition of unity (oracle).

Test infrastructure only.  Follows Section 2.2 (hierarchical decomposition)
and the partition-of-unity definition of Section 2.3.

Readings of the paper taken here (the paper is silent on them):
  * Fine level: the elements are split into P_d contiguous blocks per axis,
    floor(N_d / P_d) elements each, the first N_d mod P_d blocks one element
    longer; each block is then extended by `overlap` element layers, clipped
    to the domain (Section 2.2, step 1, with a box partition in place of the
    graph partitioner).
  * Coarse levels: the level-(l+1) subdomain indices are grouped into
    non-overlapping boxes of `group` children per axis with the same split
    rule (Section 2.2, step 2; Fig. 1 uses no overlap on coarse levels);
    T_{h,l,i} is the union of the children's element sets.
  * Partition of unity on the fine level: chi_i(x) = 0 at nodes of
    closure(Omega_i) whose hat function is not supported in closure(Omega_i)
    (these are the nodes on the internal boundary and its closure), and
    1 / N(x) otherwise, N(x) the number of subdomains for which x is such an
    interior node.  chi_i acts on nodal values (interpolation of chi_i v).
"""
import numpy as np


def split_axis(N, P):
    """Contiguous split of range(N) into P blocks; returns list of (start, end)."""
    base, rem = divmod(N, P)
    out, s = [], 0
    for p in range(P):
        e = s + base + (1 if p < rem else 0)
        out.append((s, e))
        s = e
    return out


class FineSubdomain:
    """Element box of one overlapping fine subdomain and its node sets."""

    def __init__(self, mesh, ext, core):
        self.mesh = mesh
        self.ext = ext        # per axis (start, end) element range, end exclusive
        self.core = core      # non-overlapping element range
        dim = mesh.dim
        # element mask
        coords = mesh.element_coords()
        m = np.ones(mesh.num_elements, dtype=bool)
        for d in range(dim):
            m &= (coords[:, d] >= ext[d][0]) & (coords[:, d] < ext[d][1])
        self.element_mask = m
        # Neumann space: all non-Dirichlet nodes of closure(Omega_i)
        self.neumann_box = []
        self.dirichlet_box = []
        for d in range(dim):
            lo, hi = ext[d][0], ext[d][1]                    # node range [lo, hi]
            nlo, nhi = max(lo, mesh.unknown_lo[d]), min(hi, mesh.unknown_hi[d])
            self.neumann_box.append((nlo, nhi))
            # interior nodes: hat support inside closure(Omega_i)
            dlo = lo if lo == 0 else lo + 1
            dhi = hi if hi == mesh.n[d] else hi - 1
            self.dirichlet_box.append((max(dlo, mesh.unknown_lo[d]), min(dhi, mesh.unknown_hi[d])))

    @staticmethod
    def _box_nodes(mesh, box):
        grids = np.meshgrid(*[np.arange(lo, hi + 1) for lo, hi in box], indexing="ij")
        # lexicographic, x fastest: transpose so that x varies fastest in ravel
        flat = mesh.node_index([g.transpose() for g in grids])
        return np.asarray(flat).ravel()

    def neumann_nodes(self):
        return self._box_nodes(self.mesh, self.neumann_box)

    def dirichlet_nodes(self):
        return self._box_nodes(self.mesh, self.dirichlet_box)


def fine_subdomain(mesh, parts, overlap, pidx):
    """Fine subdomain with grid index pidx (x fastest): its core element block
    of the box split, extended by `overlap` layers and clipped (Section 2.2)."""
    core = [split_axis(mesh.n[d], parts[d])[pidx[d]] for d in range(mesh.dim)]
    ext = [(max(0, c[0] - overlap), min(mesh.n[d], c[1] + overlap)) for d, c in enumerate(core)]
    return FineSubdomain(mesh, ext, core)


def pou_counts(mesh, subs):
    """N(x): the number of subdomains in `subs` for which node x is interior
    (its hat function supported in the closed subdomain)."""
    counts = np.zeros(mesh.num_nodes)
    for s in subs:
        counts[s.dirichlet_nodes()] += 1.0
    return counts


def pou_chi(mesh, sub, counts):
    """chi of `sub` on its Neumann nodes: 1 / N(x) at its interior nodes, 0 elsewhere."""
    nn = sub.neumann_nodes()
    interior = np.zeros(mesh.num_nodes, dtype=bool)
    interior[sub.dirichlet_nodes()] = True
    return np.where(interior[nn], 1.0 / np.maximum(counts[nn], 1.0), 0.0)


class Decomposition:
    """Fine subdomains plus the coarse grouping for `levels` levels.

    Level indices follow the paper: L = levels - 1 is the finest level, level 0
    is the single coarsest space.  `members[l][i]` lists the level-(l+1)
    subdomains forming level-l subdomain i (0 < l < L); `element_mask[l][i]`
    is the element set T_{h,l,i}.
    """

    def __init__(self, mesh, parts, overlap, levels, group):
        assert levels >= 2
        assert overlap >= 1, "the partition of unity needs overlap >= 1"
        self.mesh = mesh
        self.parts = tuple(parts)
        self.overlap = overlap
        self.levels = levels
        self.L = levels - 1
        dim = mesh.dim
        self.fine = []
        self.fine_grid = []
        for pidx in np.ndindex(*[parts[d] for d in reversed(range(dim))]):
            pidx = tuple(reversed(pidx))                     # x fastest
            self.fine.append(fine_subdomain(mesh, parts, overlap, pidx))
            self.fine_grid.append(pidx)
        # coarse grouping
        self.grid_shape = {self.L: tuple(parts)}
        self.members = {}
        self.element_mask = {self.L: [s.element_mask for s in self.fine]}
        self.grid_index = {self.L: list(self.fine_grid)}
        for l in range(self.L - 1, 0, -1):
            child_shape = self.grid_shape[l + 1]
            shape = tuple(max(1, child_shape[d] // group[d]) for d in range(dim))
            gsplit = [split_axis(child_shape[d], shape[d]) for d in range(dim)]
            mem, masks, gidx = [], [], []
            for q in np.ndindex(*[shape[d] for d in reversed(range(dim))]):
                q = tuple(reversed(q))
                ranges = [range(*gsplit[d][q[d]]) for d in range(dim)]
                kids = []
                for c in np.ndindex(*[len(r) for r in reversed(ranges)]):
                    c = tuple(reversed(c))
                    cidx = [ranges[d][c[d]] for d in range(dim)]
                    flat, stride = 0, 1
                    for d in range(dim):
                        flat += cidx[d] * stride
                        stride *= child_shape[d]
                    kids.append(flat)
                kids.sort()
                mem.append(kids)
                mk = np.zeros(mesh.num_elements, dtype=bool)
                for k in kids:
                    mk |= self.element_mask[l + 1][k]
                masks.append(mk)
                gidx.append(q)
            self.grid_shape[l] = shape
            self.members[l] = mem
            self.element_mask[l] = masks
            self.grid_index[l] = gidx

    def num_subdomains(self, l):
        return len(self.element_mask[l])

    def partition_of_unity(self):
        """chi_i as arrays over each subdomain's Neumann nodes (fine level)."""
        counts = pou_counts(self.mesh, self.fine)
        return [pou_chi(self.mesh, s, counts) for s in self.fine], counts

    def neighbours(self, l, i):
        """Level-(l+1) subdomains j not in J_{l,i} with T_{l+1,j} meeting T_{l,i} (Section 4.2)."""
        own = set(self.members[l][i])
        mask = self.element_mask[l][i]
        out = []
        for j, mj in enumerate(self.element_mask[l + 1]):
            if j in own:
                continue
            if np.any(mj & mask):
                out.append(j)
        return out
