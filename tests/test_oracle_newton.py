"""Pins of the oracle's coupled step (Sec. 2.4): the assembled Jacobian of the
reduced system (fluid + C W D C^T + Dirichlet rows) against central
differences of the coupled residual, the coupling operator against the
interpolation it is built from, and Newton's quadratic convergence."""
import numpy as np
import pytest

from paper_2601_08266_gb300 import inputs


def small_problem(oracle, N=4, m=60, seed=0, k_s=3.0, dt=0.5):
    from oracle import newton
    core = oracle.core
    grid = core.Grid(N)
    n = grid.n_nodes
    rng = np.random.default_rng(seed)
    phys = dict(rho=1.0, mu=0.05, dt=dt, rho_inf=0.5, has_s=True)
    Vn = rng.normal(size=(n, 4))
    An = rng.normal(size=(n, 4))
    s = rng.uniform(1.0, 3.0, n)
    f = rng.normal(size=(n, 4))
    X = inputs.ball_points(m, seed=seed + 1, radius=0.35)
    elem, xi, _ = core.locate(grid, X)
    w = rng.uniform(0.5, 1.5, m)
    X_nodes = grid.node_coords()
    bnd = np.any((X_nodes < 1e-12) | (X_nodes > 1 - 1e-12), axis=1)
    mask = np.zeros((n, 4), dtype=bool)
    mask[bnd, :3] = True
    mask[0, 3] = True
    yD = rng.normal(size=(n, 4))
    P = newton.Problem(grid, phys, Vn, An, f=f, s=s, mask=mask, yD=yD, points=(elem, xi, w),
                       solid=dict(drho=0.7, k=k_s, g=(0.0, 0.0, -9.81)))
    y = 3.0 * rng.normal(size=(n, 4))
    return P, y


def test_coupled_jacobian_matches_central_differences(oracle):
    P, y = small_problem(oracle)
    J = P.jacobian(y)
    rng = np.random.default_rng(5)
    x = rng.normal(size=y.shape)
    Jx = (J @ x.ravel()).reshape(y.shape)
    errs = []
    for eps in (1e-1, 1e-2, 1e-3):
        d = (P.residual(y + eps * x) - P.residual(y - eps * x)) / (2 * eps)
        errs.append(np.linalg.norm(d - Jx) / np.linalg.norm(Jx))
    assert errs[2] < 1e-8
    assert errs[0] > 1e-7 and 70 < errs[0] / errs[1] < 130


def test_solid_block_is_spread_of_interp(oracle):
    """The solid part of the Jacobian equals C W D C^T built from the oracle's
    own interpolation and spreading (Eq. nodal_solid_velo, fsi_constraint_matrix)."""
    from oracle import newton, timeint
    P, y = small_problem(oracle, k_s=0.0)
    core = oracle.core
    elem, xi, w = P.points
    U, A = P.stage(y)
    Jf = newton.assemble(P.grid, P.phys, U, A, P.c_a, P.c_v, f=P.f)
    x = np.random.default_rng(2).normal(size=y.shape)
    Js = P.jacobian(y) @ x.ravel() - Jf @ x.ravel()
    u = core.interp(P.grid, elem, xi, x)
    ref = core.spread(P.grid, elem, xi, 0.7 * u, w=w)
    ref[P.mask] = 0.0
    got = Js.reshape(y.shape)
    got[P.mask] = 0.0
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_coupled_newton_converges_quadratically(oracle):
    from oracle import newton
    P, y = small_problem(oracle)
    y0 = np.where(P.mask, P.yD, 0.0)
    y, hist = newton.newton(P, y0, rtol=1e-13, max_iter=12)
    h = np.array(hist)
    assert h[-1] <= 1e-13 * h[0]
    k = np.flatnonzero(h > 1e-10 * h[0])
    if len(k) >= 3:
        r = np.log(h[k[-1] + 1] / h[k[-1]]) / np.log(h[k[-1]] / h[k[-1] - 1])
        assert r > 1.5, h
