"""Pins of the oracle's P1 pressure operator K + kappa M on tetrahedral meshes
(the pressure Schur approximation of the block preconditioner, Sec. 2.4):
the textbook element matrices of the unit right tetrahedron, and closed forms
of the stiffness and mass matrices on linear fields over the unit box."""
import numpy as np
import pytest

from paper_2601_08266_gb300 import inputs


@pytest.fixture(scope="module")
def tet():
    from oracle import tet as t
    return t


@pytest.fixture(scope="module")
def mesh(tet):
    X, T = inputs.tet_box_mesh((5, 4, 6), seed=11, perturb=0.25)
    return tet.TetMesh(X, T)


def dense(A):
    return A.toarray()


def test_unit_right_tetrahedron(tet):
    X = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    m = tet.TetMesh(X, np.array([[0, 1, 2, 3]]))
    K = dense(tet.pressure_operator(m, 0.0))
    M = dense(tet.pressure_operator(m, 1.0)) - K
    K_ref = np.array([[3.0, -1, -1, -1], [-1, 1, 0, 0], [-1, 0, 1, 0], [-1, 0, 0, 1]]) / 6.0
    M_ref = (np.ones((4, 4)) + np.eye(4)) / 120.0
    assert np.allclose(K, K_ref, rtol=0, atol=1e-15)
    assert np.allclose(M, M_ref, rtol=0, atol=1e-16)
    # corner order does not matter
    m2 = tet.TetMesh(X, np.array([[2, 0, 3, 1]]))
    assert np.allclose(dense(tet.pressure_operator(m2, 1.0)), K_ref + M_ref, rtol=0, atol=1e-15)


def test_stiffness_annihilates_constants_and_measures_linear_gradients(tet, mesh):
    K = tet.pressure_operator(mesh, 0.0)
    X = mesh.X
    assert np.abs(K @ np.ones(mesh.n_nodes)).max() < 1e-13 * np.abs(K.data).max()
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    rng = np.random.default_rng(4)
    for _ in range(3):
        g = rng.normal(size=3)
        u = X @ g
        # integral of |grad u|^2 over the unit box
        assert u @ (K @ u) == pytest.approx(g @ g, rel=1e-12)
        # interior rows of K u vanish for linear u (no boundary term)
        assert np.abs((K @ u)[inner]).max() < 1e-12 * np.abs(g).max()


def test_mass_integrates_products_of_linear_fields(tet, mesh):
    M = tet.pressure_operator(mesh, 1.0) - tet.pressure_operator(mesh, 0.0)
    one = np.ones(mesh.n_nodes)
    x, y, z = mesh.X.T
    assert one @ (M @ one) == pytest.approx(1.0, rel=1e-12)
    assert x @ (M @ x) == pytest.approx(1.0 / 3.0, rel=1e-12)
    assert x @ (M @ y) == pytest.approx(1.0 / 4.0, rel=1e-12)
    assert (1 + 2 * z) @ (M @ (y - z)) == pytest.approx(-1.0 / 6.0, rel=1e-12)


def test_symmetric_positive_definite(tet, mesh):
    A = dense(tet.pressure_operator(mesh, (np.pi / 2.0) ** 2))
    assert np.abs(A - A.T).max() < 1e-15 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_eliminated_nodes_keep_only_their_diagonal(tet, mesh):
    kappa = 0.7
    X = mesh.X
    el = np.any(X > 1 - 1e-12, axis=1) & (X[:, 1] > 0.3)
    A = dense(tet.pressure_operator(mesh, kappa))
    B = dense(tet.pressure_operator(mesh, kappa, eliminated=el))
    idx = np.flatnonzero(el)
    assert idx.size > 0
    assert np.array_equal(np.diag(B), np.diag(A))
    off = ~np.eye(mesh.n_nodes, dtype=bool)
    assert not np.any(B[idx][:, ~el]) and not np.any(B[:, idx][~el])
    assert np.count_nonzero(B[np.ix_(idx, idx)] * off[np.ix_(idx, idx)]) == 0
    keep = ~el
    assert np.array_equal(B[np.ix_(keep, keep)], A[np.ix_(keep, keep)])
