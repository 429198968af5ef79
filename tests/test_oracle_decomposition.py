"""Pins of the oracle's decomposition and partition of unity (Sections 2.2, 2.3, 3.1)."""
import numpy as np
import pytest

from oracle import decomposition as dd
from oracle import fem


def test_split_axis():
    assert dd.split_axis(10, 3) == [(0, 4), (4, 7), (7, 10)]
    assert dd.split_axis(64, 4) == [(0, 16), (16, 32), (32, 48), (48, 64)]


@pytest.mark.parametrize("n,parts,overlap,faces", [
    ((16, 16), (4, 4), 1, 0b1), ((19, 13), (3, 2), 2, 0b1), ((9, 8, 7), (2, 2, 2), 1, 0b11),
    ((16, 16), (4, 4), 2, 0)])
def test_partition_of_unity(n, parts, overlap, faces):
    """sum_i e chi_i r_i v = v for all v and chi_i = 0 on the internal boundary (Def. in Section 2.3)."""
    mesh = fem.Mesh(n, faces)
    dec = dd.Decomposition(mesh, parts, overlap, 2, (2,) * len(n))
    chis, counts = dec.partition_of_unity()
    total = np.zeros(mesh.num_nodes)
    unk = mesh.node_to_unknown() >= 0
    for s, chi in zip(dec.fine, chis):
        total[s.neumann_nodes()] += chi
        # chi vanishes exactly where the hat function leaves closure(Omega_i)
        coords = np.array(np.unravel_index(s.neumann_nodes(), mesh.nodes_per_axis[::-1]))[::-1]
        on_internal = np.zeros(len(chi), dtype=bool)
        for d in range(mesh.dim):
            lo, hi = s.ext[d]
            on_internal |= (coords[d] == lo) & (lo > 0)
            on_internal |= (coords[d] == hi) & (hi < mesh.n[d])
        assert np.all(chi[on_internal] == 0.0)
        assert np.all(chi[~on_internal] > 0.0)
    assert np.allclose(total[unk], 1.0)


def test_dirichlet_matrix_is_principal_block_of_neumann():
    """For interior nodes all adjacent elements are in T_i, so A_i = R A R^T = Abar_i restricted."""
    mesh = fem.Mesh((12, 10), 0b1)
    kap = np.random.default_rng(0).lognormal(0, 1, mesh.num_elements)
    dec = dd.Decomposition(mesh, (3, 2), 2, 2, (3, 2))
    A = fem.assemble_system(mesh, kap)
    n2u = mesh.node_to_unknown()
    An = fem.assemble_neumann(mesh, kap)
    for s in dec.fine:
        Abar = fem.assemble_neumann(mesh, kap, s.element_mask)
        dn = s.dirichlet_nodes()
        assert np.allclose(Abar[dn][:, dn].toarray(), A[n2u[dn]][:, n2u[dn]].toarray())
        # the Neumann matrix differs from the global one on boundary nodes
        nn = s.neumann_nodes()
        assert len(nn) > len(dn)


def test_coloring_and_admissibility():
    """Def. coloring: 4 colours in 2D (x-parity, y-parity) separate subdomains
    whose Dirichlet spaces interact; every interior edge is interior to a subdomain."""
    mesh = fem.Mesh((32, 32), 0b1)
    dec = dd.Decomposition(mesh, (4, 4), 2, 2, (2, 2))
    A = fem.assemble_system(mesh, np.ones(mesh.num_elements))
    n2u = mesh.node_to_unknown()
    for i, si in enumerate(dec.fine):
        for j, sj in enumerate(dec.fine):
            if i == j:
                continue
            pi, pj = dec.fine_grid[i], dec.fine_grid[j]
            if (pi[0] % 2, pi[1] % 2) == (pj[0] % 2, pj[1] % 2):
                block = A[n2u[si.dirichlet_nodes()]][:, n2u[sj.dirichlet_nodes()]]
                assert block.nnz == 0 or np.abs(block.toarray()).max() == 0
    # admissibility: each element's interior lies in some subdomain's interior,
    # i.e. every node is interior to at least one subdomain (counts >= 1)
    _, counts = dec.partition_of_unity()
    assert counts[n2u >= 0].min() >= 1


def test_coarse_grouping():
    mesh = fem.Mesh((64, 64), 0b1)
    dec = dd.Decomposition(mesh, (8, 8), 2, 4, (2, 2))
    assert dec.grid_shape == {3: (8, 8), 2: (4, 4), 1: (2, 2)}
    assert dec.members[2][0] == [0, 1, 8, 9]
    # the groups partition the children
    for l in (2, 1):
        allk = sorted(k for m in dec.members[l] for k in m)
        assert allk == list(range(dec.num_subdomains(l + 1)))
    # a corner group of 2x2 fine subdomains sees the 5 fine neighbours of its ring
    assert sorted(dec.neighbours(2, 0)) == [2, 10, 16, 17, 18]
