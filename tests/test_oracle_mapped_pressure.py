"""Pins of the oracle's pressure operator on a mapped structured grid
(K + kappa M of the Q1 pressure space at the true node coordinates, the exact
Schur approximation of Sec. 2.4): the textbook tensor-product form on a
uniform grid, the null space and the linear patch test of K (exact with
2x2x2 Gauss points on any trilinear map), the volume and first moment the mass
matrix integrates, symmetry and semi-definiteness, and the elimination rule."""
import math

import numpy as np
import scipy.sparse as sp

from oracle import precond


def grid_coords(N, x0=(0.0, 0.0, 0.0), h=(1.0, 1.0, 1.0)):
    ax = [x0[d] + h[d] * np.arange(N[d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)


def interior(N):
    i, j, k = np.meshgrid(*(np.arange(N[d] + 1) for d in (2, 1, 0)), indexing="ij")
    k, j, i = i.ravel(), j.ravel(), k.ravel()
    return (i > 0) & (i < N[0]) & (j > 0) & (j < N[1]) & (k > 0) & (k < N[2])


def lin1d(n, h):
    """1D linear-element stiffness and mass on n elements of size h (textbook)."""
    K = sp.diags([-np.ones(n), 2 * np.ones(n + 1), -np.ones(n)], [-1, 0, 1]).tolil() / h
    M = sp.diags([np.ones(n), 4 * np.ones(n + 1), np.ones(n)], [-1, 0, 1]).tolil() * (h / 6)
    K[0, 0] = K[n, n] = 1.0 / h
    M[0, 0] = M[n, n] = h / 3
    return K.tocsr(), M.tocsr()


def perturbed(N, h, amp, seed):
    X = grid_coords(N, h=h)
    inn = interior(N)
    rng = np.random.default_rng(seed)
    X[inn] += amp * rng.uniform(-1, 1, (inn.sum(), 3)) * np.asarray(h)[None, :]
    return X


def test_uniform_grid_is_the_tensor_product_of_1d_matrices():
    N, h, kappa = (4, 3, 5), (0.3, 0.5, 0.2), 0.7
    A = precond.mapped_pressure_operator(N, grid_coords(N, x0=(1.0, -2.0, 0.5), h=h), kappa)
    (Kx, Mx), (Ky, My), (Kz, Mz) = (lin1d(N[d], h[d]) for d in range(3))
    ref = (sp.kron(Mz, sp.kron(My, Kx)) + sp.kron(Mz, sp.kron(Ky, Mx)) +
           sp.kron(Kz, sp.kron(My, Mx)) + kappa * sp.kron(Mz, sp.kron(My, Mx)))
    assert abs(A - ref).max() <= 1e-13 * abs(ref).max()
    # default shift from the bounding box
    A0 = precond.mapped_pressure_operator(N, grid_coords(N, h=h))
    L = max(N[d] * h[d] for d in range(3))
    Ak = precond.mapped_pressure_operator(N, grid_coords(N, h=h), (math.pi / (2 * L)) ** 2)
    assert abs(A0 - Ak).max() == 0.0


def test_affine_map_null_space_patch_test_and_moments():
    N = (3, 4, 2)
    B = np.array([[1.2, 0.3, -0.1], [0.2, 0.9, 0.25], [-0.15, 0.1, 1.4]])
    b = np.array([0.5, -1.0, 2.0])
    X = grid_coords(N, h=(0.5, 0.25, 0.5)) @ B.T + b
    K = precond.mapped_pressure_operator(N, X, kappa=0.0)
    M = (precond.mapped_pressure_operator(N, X, kappa=1.0) - K).tocsr()
    one = np.ones(X.shape[0])
    assert np.abs(K @ one).max() <= 1e-13 * abs(K).max()
    inn = interior(N)
    for c in (np.array([1.0, 0.0, 0.0]), np.array([0.3, -0.7, 1.1])):
        r = K @ (X @ c)
        assert np.abs(r[inn]).max() <= 1e-12 * abs(K).max()
        assert np.abs(r[~inn]).max() > 1e-6       # boundary fluxes remain
    vol = np.linalg.det(B) * 1.5 * 1.0 * 1.0
    assert abs(one @ M @ one - vol) <= 1e-13 * vol
    centroid = B @ np.array([0.75, 0.5, 0.5]) + b
    assert np.allclose(one @ M @ X, centroid * vol, rtol=1e-13, atol=1e-13)


def test_trilinear_map_is_exact_for_null_space_patch_test_and_volume():
    N, h = (5, 4, 6), (0.2, 0.25, 1.0 / 6)
    X = perturbed(N, h, 0.3, seed=3)
    K = precond.mapped_pressure_operator(N, X, kappa=0.0)
    M = (precond.mapped_pressure_operator(N, X, kappa=1.0) - K).tocsr()
    one = np.ones(X.shape[0])
    assert np.abs(K @ one).max() <= 1e-12 * abs(K).max()
    inn = interior(N)
    r = K @ (X @ np.array([0.4, 1.0, -0.6]))
    assert np.abs(r[inn]).max() <= 1e-11 * abs(K).max()
    # only interior nodes moved: the elements still tile the unit cube
    assert abs(one @ M @ one - 1.0) <= 1e-13
    assert np.allclose(one @ M @ X, [0.5, 0.5, 0.5], rtol=0, atol=1e-13)
    # symmetric positive semi-definite K, positive definite K + kappa M
    A = precond.mapped_pressure_operator(N, X).toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    assert np.linalg.eigvalsh(K.toarray()).min() >= -1e-12
    assert np.linalg.eigvalsh(A).min() > 0
    # a distorted map changes the operator away from the nominal box
    U = precond.mapped_pressure_operator(N, grid_coords(N, h=h))
    assert abs(A - U.toarray()).max() > 1e-3 * np.abs(A).max()


def test_elimination_keeps_the_diagonal_only():
    N, h = (3, 3, 3), (1 / 3,) * 3
    X = perturbed(N, h, 0.2, seed=5)
    el = ~interior(N)
    A = precond.mapped_pressure_operator(N, X).toarray()
    Ae = precond.mapped_pressure_operator(N, X, eliminated=el).toarray()
    keep = ~el
    assert np.array_equal(Ae[np.ix_(keep, keep)], A[np.ix_(keep, keep)])
    assert np.array_equal(np.diag(Ae), np.diag(A))
    off = Ae - np.diag(np.diag(Ae))
    assert not off[el].any() and not off[:, el].any()
