"""Pins of the preconditioner oracle (oracle/precond.py): the Q1 pressure
operator against exact integrals, the transfer operators against trilinear
reproduction and the Galerkin property, the smoother against the Chebyshev
polynomial, the spectrum bound against dense eigenvalues, and the V-cycle's
grid-independent contraction."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import precond as pc


def nodes(level):
    ax = [np.arange(level.N[d] + 1) * level.h[d] for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    return X.ravel(), Y.ravel(), Z.ravel()


@pytest.mark.parametrize("N,h", [((4, 4, 4), (0.25, 0.25, 0.25)), ((3, 5, 2), (0.2, 0.1, 0.3))])
def test_stiffness_and_mass_match_exact_integrals(N, h):
    L = pc.Level(N, h)
    _, K, M = pc.assemble(L)
    X, Y, Z = nodes(L)
    Lx, Ly, Lz = (N[d] * h[d] for d in range(3))
    vol = Lx * Ly * Lz
    one = np.ones(L.n)
    assert np.abs(K @ one).max() < 1e-12                       # constants in the kernel
    assert one @ (M @ one) == pytest.approx(vol, rel=1e-13)
    u = 2.0 * X - 3.0 * Y + 0.5 * Z + 1.0                      # |grad u|^2 = 13.25
    assert u @ (K @ u) == pytest.approx(13.25 * vol, rel=1e-12)
    w = X * Y * Z                                              # trilinear: in the Q1 space
    # int |grad(xyz)|^2 = int y^2 z^2 + x^2 z^2 + x^2 y^2 over the box
    exact_k = (Lx * Ly ** 3 * Lz ** 3 + Lx ** 3 * Ly * Lz ** 3 + Lx ** 3 * Ly ** 3 * Lz) / 9.0
    assert w @ (K @ w) == pytest.approx(exact_k, rel=1e-12)
    assert w @ (M @ w) == pytest.approx(Lx ** 3 * Ly ** 3 * Lz ** 3 / 27.0, rel=1e-12)


def test_prolongation_reproduces_trilinear_fields():
    fine = pc.Level((8, 6, 4), (0.1, 0.2, 0.25))
    coarse = pc.Level((4, 3, 2), (0.2, 0.4, 0.5))
    P = pc.prolongation(fine, coarse)
    f = lambda x, y, z: 1 + 2 * x - y + 3 * z + x * y - y * z + 2 * x * y * z - 0.5 * x * z
    uc = f(*nodes(coarse))
    uf = f(*nodes(fine))
    assert np.abs(P @ uc - uf).max() < 1e-13
    assert np.allclose(P.sum(axis=1), 1.0)                     # partition of unity


@pytest.mark.parametrize("N", [(8, 8, 8), (12, 6, 4)])
def test_galerkin_property_of_the_hierarchy(N):
    h = tuple(1.0 / v for v in N)
    mg = pc.MultigridOracle(N, h)
    assert len(mg.levels) >= 2
    for l in range(len(mg.levels) - 1):
        G = (mg.P[l].T @ mg.A[l] @ mg.P[l]).toarray()
        assert np.abs(G - mg.A[l + 1].toarray()).max() < 1e-12 * np.abs(G).max()


def test_hierarchy_rule():
    assert [L.N for L in pc.hierarchy((128,) * 3, (1 / 128,) * 3)] == [
        (128,) * 3, (64,) * 3, (32,) * 3, (16,) * 3, (8,) * 3, (4,) * 3]
    assert [L.N for L in pc.hierarchy((14,) * 3, (1 / 14,) * 3)] == [(14,) * 3, (7,) * 3]
    assert [L.N for L in pc.hierarchy((6, 5, 7), (0.2, 0.1, 0.1))] == [(6, 5, 7)]
    assert pc.kappa_of((8, 4, 4), (0.1, 0.3, 0.3)) == pytest.approx((math.pi / 2.4) ** 2)


@pytest.mark.parametrize("N,h", [((4, 4, 4), (0.25,) * 3), ((6, 5, 7), (0.2, 0.1, 0.1)),
                                 ((8, 4, 4), (0.1, 0.3, 0.3)), ((2, 2, 2), (0.5,) * 3)])
def test_spectrum_bound_covers_and_is_tight(N, h):
    kap = pc.kappa_of(N, h)
    A = pc.assemble(pc.Level(N, h), kap)[0].toarray()
    lam = sla.eigvalsh(A, np.diag(np.diag(A)))
    hi = pc.spectrum_bound(h, kap)
    assert lam.max() <= hi
    assert lam.max() >= hi / 1.1 * 0.95


def test_chebyshev_error_is_the_scaled_chebyshev_polynomial():
    lam = np.linspace(0.05, 1.6, 37)
    A = np.diag(lam)
    b = np.random.default_rng(1).normal(size=lam.size)
    lo, hi = 0.4, 1.6
    theta, delta = (hi + lo) / 2, (hi - lo) / 2

    def T(m, t):     # Chebyshev polynomial of the first kind, any real t
        return np.cos(m * np.arccos(t)) if np.all(np.abs(t) <= 1) else np.where(
            np.abs(t) <= 1, np.cos(m * np.arccos(np.clip(t, -1, 1))),
            np.cosh(m * np.arccosh(np.maximum(np.abs(t), 1))) * np.sign(t) ** m)

    for m in (1, 2, 3, 5):
        x = pc.chebyshev(A, np.ones(lam.size), b, np.zeros(lam.size), m, lo, hi)
        e0 = b / lam
        p = T(m, (theta - lam) / delta) / T(m, theta / delta)
        assert np.allclose(e0 - x, p * e0, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("N", [8, 16, 14, 12])
def test_vcycle_contracts_independently_of_the_grid(N):
    mg = pc.MultigridOracle(N)
    A = mg.A[0]
    rng = np.random.default_rng(N)
    b = rng.normal(size=A.shape[0])
    xs = spla.spsolve(A.tocsc(), b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(4):
        x = x + mg.vcycle(b - A @ x)
        e = x - xs
        errs.append(math.sqrt(e @ (A @ e)))
    rates = [errs[i + 1] / errs[i] for i in range(3)]
    assert max(rates) < 0.08, rates


def test_vcycle_is_a_fixed_symmetric_linear_operator():
    mg = pc.MultigridOracle((8, 8, 8))
    n = mg.A[0].shape[0]
    rng = np.random.default_rng(5)
    u, v = rng.normal(size=n), rng.normal(size=n)
    Vu, Vv = mg.vcycle(u), mg.vcycle(v)
    assert np.allclose(mg.vcycle(2 * u - 3 * v), 2 * Vu - 3 * Vv, rtol=1e-12, atol=1e-12)
    assert u @ Vv == pytest.approx(v @ Vu, rel=1e-10)
    assert u @ Vu > 0


def test_sigma_is_the_generalized_alpha_chain_ratio():
    # rho_inf = 0.5: alpha_m = 5/6, alpha_f = gamma = 2/3 -> sigma = 0.5333 dt / rho
    assert pc.sigma_of(1.0, 1e-3) == pytest.approx(0.16 / 0.3 * 1e-3)
    assert pc.sigma_of(2.0, 1e-2) == pytest.approx(0.16 / 0.3 * 1e-2 / 2.0)


def test_faces_from_mask_finds_the_free_faces():
    N = (6, 5, 4)
    L = pc.Level(N, (1.0, 1.0, 1.0))
    k, j, i = np.indices((N[2] + 1, N[1] + 1, N[0] + 1)).reshape(3, -1)
    mask = np.zeros((L.n, 4), dtype=bool)
    walls = (j == 0) | (j == N[1]) | (k == 0) | (k == N[2])
    mask[walls | (i == 0), :3] = True          # no-slip walls and an inflow at x = 0
    assert pc.faces_from_mask(N, mask) == (0, 1, 0, 0, 0, 0)
    assert pc.faces_from_mask(N, np.zeros((L.n, 4), bool)) == (1,) * 6
    assert pc.faces_from_mask(N, np.ones((L.n, 4), bool)) == (0,) * 6


def test_eliminated_faces_keep_galerkin_and_contraction():
    faces = (0, 1, 0, 0, 1, 0)
    mg = pc.MultigridOracle((16, 16, 16), faces=faces)
    for l in range(len(mg.levels) - 1):
        keep_f, keep_c = ~mg.dirn[l], ~mg.dirn[l + 1]
        Pi = mg.P[l][keep_f][:, keep_c]
        G = (Pi.T @ mg.A[l][keep_f][:, keep_f] @ Pi).toarray()
        Ac = mg.A[l + 1][keep_c][:, keep_c].toarray()
        assert np.abs(G - Ac).max() < 1e-12 * np.abs(Ac).max()
        # the eliminated rows are decoupled diagonal rows
        Ad = mg.A[l][mg.dirn[l]]
        assert Ad.nnz == int(mg.dirn[l].sum())
    A = mg.A[0]
    b = np.random.default_rng(4).normal(size=A.shape[0])
    xs = spla.spsolve(A.tocsc(), b)
    x = np.zeros_like(b)
    errs = []
    for _ in range(4):
        x = x + mg.vcycle(b - A @ x)
        e = x - xs
        errs.append(math.sqrt(e @ (A @ e)))
    assert max(errs[i + 1] / errs[i] for i in range(3)) < 0.1


@pytest.mark.parametrize("N", [6, 10])
def test_schur_complement_is_spectrally_equivalent_to_the_approximation(N):
    """The pressure Schur complement of the oracle's assembled Jacobian (a
    channel with leaflets, dt = 1e-3) against sigma (K + kappa M) with the
    free outflow face eliminated: eigenvalue ratios stay in a fixed band as h
    shrinks (without the elimination the largest grows like 1/h)."""
    from oracle import core, newton
    from paper_2601_08266_gb300 import inputs
    grid = core.Grid(N)
    n = grid.n_nodes
    X, Y, Z = grid.node_coords().T
    wall = (Y < 1e-12) | (Y > 1 - 1e-12) | (Z < 1e-12) | (Z > 1 - 1e-12)
    inflow = (X < 1e-12) & ~wall
    mask = np.zeros((n, 4), bool)
    mask[wall | inflow, :3] = True
    rng = np.random.default_rng(2)
    Vn = np.zeros((n, 4))
    Vn[:, 0] = 16 * Y * (1 - Y) * Z * (1 - Z)
    Vn[:, :3] += 0.05 * rng.normal(size=(n, 3))
    Vn[mask] = 0.0
    m = 800
    e, xi, _ = core.locate(grid, inputs.leaflet_points(m, seed=5))
    dt = 1e-3
    P = newton.Problem(grid, dict(rho=1.0, mu=1e-3, dt=dt, rho_inf=0.5), Vn, np.zeros((n, 4)),
                       mask=mask, yD=np.zeros((n, 4)), points=(e, xi, np.full(m, 0.024 / m)),
                       solid=dict(drho=0.5, k=0.0, g=(0, 0, 0)))
    J = P.jacobian(np.zeros((n, 4))).toarray()
    vel = np.arange(4 * n) % 4 < 3
    S = J[np.ix_(~vel, ~vel)] - J[np.ix_(~vel, vel)] @ np.linalg.solve(
        J[np.ix_(vel, vel)], J[np.ix_(vel, ~vel)])
    faces = pc.faces_from_mask((N,) * 3, mask)
    assert faces == (0, 1, 0, 0, 0, 0)
    sig = pc.sigma_of(1.0, dt)
    kap = pc.kappa_of((N,) * 3, (1.0 / N,) * 3)
    lev = pc.Level((N,) * 3, (1.0 / N,) * 3)
    ev = sla.eigvals(S, sig * pc.assemble(lev, kap, faces)[0].toarray()).real
    assert ev.min() > 0.4 and ev.max() < 2.0, (ev.min(), ev.max())
    ev0 = sla.eigvals(S, sig * pc.assemble(lev, kap)[0].toarray()).real
    assert ev0.max() > 3.0 * ev.max()          # the Neumann-only approximation is far off
