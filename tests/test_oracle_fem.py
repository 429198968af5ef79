"""Pins of the oracle's Q1 assembly (Section 3.4, forms a_tau, a_h, l).

Every expected value here comes from mathematics independent of the oracle's
code path: a second derivation of the element matrix, exact integrals of
polynomials, and the exact solution of a 1D boundary value problem to which
the 2D discrete problem reduces.
"""
import numpy as np
import pytest

from oracle import fem


def test_q1_2d_closed_form_matches_quadrature():
    # two independent derivations: tensor-product closed form vs Gauss quadrature
    for hx, hy in [(1.0, 1.0), (0.25, 0.5), (1 / 64, 1 / 64)]:
        A = fem.q1_element_matrix_quadrature((hx, hy), np.eye(2))
        B = fem.q1_element_matrix_2d_scalar(1.0, hx, hy)
        assert np.allclose(A, B, rtol=0, atol=1e-14 * np.abs(B).max())


def test_q1_2d_square_element_values():
    # on a square the Laplacian element matrix is independent of h:
    # diagonal 2/3, edge neighbours -1/6, diagonal neighbour -1/3
    A = fem.q1_element_matrix_quadrature((0.1, 0.1), np.eye(2))
    # local order x fastest: 0=(0,0) 1=(1,0) 2=(0,1) 3=(1,1)
    assert np.isclose(A[0, 0], 2 / 3)
    assert np.isclose(A[0, 1], -1 / 6) and np.isclose(A[0, 2], -1 / 6)
    assert np.isclose(A[0, 3], -1 / 3)


@pytest.mark.parametrize("dim", [2, 3])
def test_element_matrix_kernel_and_linear_energy(dim):
    rng = np.random.default_rng(1)
    h = rng.uniform(0.1, 1.0, dim)
    M = rng.standard_normal((dim, dim))
    K = M @ M.T + dim * np.eye(dim)
    A = fem.q1_element_matrix_quadrature(h, K)
    assert np.allclose(A, A.T)
    assert np.allclose(A @ np.ones(2 ** dim), 0.0, atol=1e-12)       # constants in kernel
    # energy of the linear function u = g . x equals g^T K g * |tau| exactly
    g = rng.standard_normal(dim)
    corners = np.array([[(a >> d) & 1 for d in range(dim)] for a in range(2 ** dim)]) * h
    u = corners @ g
    assert np.isclose(u @ A @ u, g @ K @ g * np.prod(h), rtol=1e-12)
    w = np.linalg.eigvalsh(A)
    assert w[0] > -1e-12 and np.sum(w < 1e-10) == 1               # kernel exactly 1-D


def test_tensor_coefficient_reduces_to_scalar():
    mesh = fem.Mesh((3, 2, 2), 0)
    kap = np.linspace(1, 2, mesh.num_elements)
    comps = np.zeros((mesh.num_elements, 6))
    comps[:, 0] = comps[:, 1] = comps[:, 2] = kap
    assert np.allclose(fem.element_matrices(mesh, kap), fem.element_matrices(mesh, comps))


def test_neumann_matrix_annihilates_constants():
    mesh = fem.Mesh((7, 5), 0)
    kap = np.random.default_rng(0).lognormal(0, 2, mesh.num_elements)
    A = fem.assemble_neumann(mesh, kap)
    assert np.abs(A @ np.ones(mesh.num_nodes)).max() < 1e-12 * kap.max()


def test_load_vector_integrates_to_area():
    for n, faces in [((8, 8), 0), ((8, 6), 0b1), ((4, 4, 4), 0)]:
        mesh = fem.Mesh(n, faces)
        b = fem.load_vector(mesh)
        if faces == 0:
            assert np.isclose(b.sum(), 1.0)
        else:
            # nodes on x=0 removed: a half-column of width h/2 per row removed
            assert np.isclose(b.sum(), 1.0 - 0.5 / n[0])


@pytest.mark.parametrize("N,M", [(8, 8), (16, 5), (32, 32)])
def test_manufactured_solution_is_nodally_exact(N, M):
    """-u'' = 1, u(0)=0, u'(1)=0 has u = x - x^2/2.

    With kappa = 1, Dirichlet on x = 0 only and Neumann elsewhere, the Q1
    system for a y-independent nodal vector reduces (stiffness = K_x (x) M_y
    + M_x (x) K_y, K_y 1 = 0) to 1D linear finite elements, which are nodally
    exact for this problem.
    """
    mesh = fem.Mesh((N, M), 0b1)
    A = fem.assemble_system(mesh, np.ones(mesh.num_elements))
    b = fem.load_vector(mesh)
    import scipy.sparse.linalg as spla
    u = spla.spsolve(A.tocsc(), b)
    x = np.tile(np.arange(1, N + 1) / N, M + 1)
    assert np.abs(u - (x - 0.5 * x * x)).max() < 1e-12


@pytest.mark.parametrize("faces,axis", [(0b11, 0), (0b1100, 1)])
def test_manufactured_solution_two_dirichlet_faces(faces, axis):
    """-u'' = 1 along one axis with u = 0 on both of its faces has
    u = t (1 - t) / 2; with kappa = 1 and Neumann on the other faces the Q1
    system reduces to 1D linear elements as above, which are nodally exact.
    Pins the unknown numbering and the load vector with Dirichlet faces at
    x_d = 1 as well as x_d = 0."""
    N, M = (10, 7) if axis == 0 else (7, 10)
    mesh = fem.Mesh((N, M), faces)
    A = fem.assemble_system(mesh, np.ones(mesh.num_elements))
    b = fem.load_vector(mesh)
    import scipy.sparse.linalg as spla
    u = spla.spsolve(A.tocsc(), b)
    sx, sy = mesh.unknown_shape
    ix, iy = np.meshgrid(np.arange(sx) + mesh.unknown_lo[0], np.arange(sy) + mesh.unknown_lo[1], indexing="xy")
    t = (ix / N if axis == 0 else iy / M).ravel()
    assert np.abs(u - 0.5 * t * (1 - t)).max() < 1e-12


def test_unknown_numbering_is_lexicographic():
    mesh = fem.Mesh((4, 3), 0b1 | 0b1000)         # x=0 and y=1 Dirichlet
    n2u = mesh.node_to_unknown()
    assert mesh.unknown_shape == (4, 3)
    # node (ix=1, iy=0) is unknown 0, (ix=4, iy=2) is the last, y=3 removed
    assert n2u[mesh.node_index((1, 0))] == 0
    assert n2u[mesh.node_index((4, 2))] == 11
    assert n2u[mesh.node_index((2, 3))] == -1
    assert n2u[mesh.node_index((0, 1))] == -1
    assert n2u[mesh.node_index((2, 1))] == 1 + 4 * 1
