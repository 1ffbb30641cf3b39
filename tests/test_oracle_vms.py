"""Pins of the oracle's VMS residual, tau parameters and Jacobian.

* tau_m / tau_c (Sec. 2.1): closed-form limits.
* residual: exact single-element integration of the inner-product VMS form
  (weakform_ref, 4x4x4 Gauss) on fields where the method's 2x2x2 rule is
  exact (linear velocity with orthogonal columns, so tau is the same at every
  method Gauss point); Galerkin part on multi-element anisotropic grids;
  the continuity row sum (divergence theorem); manufactured-solution
  convergence rates (cf. the rates of Sec. 4.1).
* Jacobian: central finite differences of the residual, O(eps^2); the PSPG
  pressure block is symmetric positive semidefinite with constant null space.
"""
import json
import math
import os

import numpy as np
import pytest

from paper_2601_08266_gb300 import inputs
import weakform_ref as wf

Q = 1.0 / math.sqrt(3.0)
GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def test_default_constants_are_the_papers(oracle):
    """C_I = 36 and C_T = 4 (Sec. 2.1) are the oracle's defaults."""
    core = oracle.core
    p = core.phys_array(dict(rho=1.0, mu=0.0, dt=0.5))
    assert p[3] == GOLDEN["C_I"]["value"]
    assert p[2] == GOLDEN["C_T"]["value"] / 0.25


def local_nodes(grid, e):
    N = grid.N
    ex, ey, ez = e % N[0], (e // N[0]) % N[1], e // (N[0] * N[1])
    out = []
    for a in range(8):
        i, j, k = ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)
        out.append(i + (N[0] + 1) * (j + (N[1] + 1) * k))
    return np.array(out)


def test_tau_closed_forms(oracle):
    core = oracle.core
    h, dt, s = 0.125, 1e-3, 4.0
    # v = 0, mu = 0: tau_M = (s C_T/dt^2)^(-1/2) = dt/(2 sqrt(s)); tau_C = 1/(tau_M tr G)
    tm, tc = core.tau([0, 0, 0], s, h, 1.0, 0.0, dt)
    assert tm == pytest.approx(dt / (2 * math.sqrt(s)), rel=1e-15)
    assert tc == pytest.approx(1.0 / (tm * 12.0 / h ** 2), rel=1e-15)
    # steady inviscid, v along x: tau_M = h/(2|v|)
    tm, _ = core.tau([3.0, 0, 0], 1.0, h, 1.0, 0.0, None)
    assert tm == pytest.approx(h / 6.0, rel=1e-15)
    # steady, v = 0, viscous: tau_M = h^2 / (nu sqrt(C_I * 48))
    tm, _ = core.tau([0, 0, 0], 1.0, h, 2.0, 0.5, None)
    assert tm == pytest.approx(h * h / (0.25 * math.sqrt(36.0 * 48.0)), rel=1e-14)
    # anisotropic cell: v.G v = 4 (vx^2/hx^2 + ...)
    tm, tc = core.tau([1.0, 2.0, 0.0], 1.0, (0.5, 0.25, 1.0), 1.0, 0.0, None)
    assert tm == pytest.approx(1.0 / math.sqrt(4 * (1 / 0.25 + 4 / 0.0625)), rel=1e-15)
    assert tc == pytest.approx(1.0 / (tm * 4 * (4 + 16 + 1)), rel=1e-15)


def _rotation(rng):
    q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    return q


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_single_element_exact_integration(oracle, seed):
    """Full VMS residual on one element vs. the inner-product form."""
    core = oracle.core
    rng = np.random.default_rng(seed)
    h = 0.37
    grid = core.Grid(1, x0=(0.1, -0.2, 0.3), h=h)
    M = _rotation(rng) @ np.diag(rng.uniform(0.5, 2.0, 3))   # orthogonal columns
    xi_nodes = np.array([[2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1]
                         for a in range(8)], dtype=float)
    U = np.zeros((8, 4))
    U[:, :3] = xi_nodes @ M.T
    U[:, 3] = rng.normal(size=8)
    A = np.zeros((8, 4))
    A[:, :3] = rng.normal(size=(8, 3))
    s = rng.uniform(1.0, 5.0)
    A[:, 3] = s
    f = rng.normal(size=(8, 4))
    rho, mu, dt = rng.uniform(0.5, 2.0), rng.uniform(0.01, 0.5), 0.05
    phys = dict(rho=rho, mu=mu, dt=dt, has_s=True)
    R = core.residual(grid, phys, U, A, f=f)
    # |v|^2 at every 2x2x2 Gauss point = Q^2 * sum of squared column norms
    vGv = (4.0 / h ** 2) * Q * Q * np.sum(M * M)
    tm = 1.0 / math.sqrt(s * (4.0 / dt ** 2 + vGv + 36.0 * (mu / rho) ** 2 * 3 * (4 / h ** 2) ** 2))
    tc = 1.0 / (tm * 3 * 4.0 / h ** 2)
    ref = wf.element_weak_form((h, h, h), U, A, f, rho, mu,
                               lambda v: np.full(len(v), tm), lambda v: np.full(len(v), tc))
    assert np.abs(R - ref).max() <= 1e-12 * np.abs(ref).max()
    # the stabilisation terms are a sizable part of the result
    gal = wf.element_weak_form((h, h, h), U, A, f, rho, mu, None, None, stab=False)
    assert np.abs(ref - gal).max() > 1e-3 * np.abs(ref).max()


def test_galerkin_multi_element_exact(oracle):
    """Plain Galerkin part, general Q1 fields, anisotropic 3x2x2 grid."""
    core = oracle.core
    rng = np.random.default_rng(5)
    grid = core.Grid((3, 2, 2), x0=(0.0, 1.0, -1.0), h=(0.3, 0.7, 0.45))
    n = grid.n_nodes
    U, A, f = rng.normal(size=(n, 4)), rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    phys = dict(rho=1.3, mu=0.2, dt=0.01)
    R = core.residual(grid, phys, U, A, f=f, stab=False)
    ref = np.zeros((n, 4))
    for e in range(grid.n_elems):
        ln = local_nodes(grid, e)
        ref[ln] += wf.element_weak_form(grid.h, U[ln], A[ln], f[ln], 1.3, 0.2, None, None,
                                        stab=False)
    assert np.abs(R - ref).max() <= 1e-13 * np.abs(ref).max()


def test_continuity_row_sum_is_total_divergence(oracle):
    """sum_A R^c_A = int div v dOmega (sum_A N_A = 1, sum_A grad N_A = 0), which by
    the divergence theorem is the boundary flux of the trilinear v."""
    core = oracle.core
    rng = np.random.default_rng(9)
    grid = core.Grid((4, 3, 2), h=(0.25, 1 / 3, 0.5))
    n = grid.n_nodes
    U, A = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    R = core.residual(grid, dict(rho=1.0, mu=0.05, dt=0.01), U, A)
    Nx, Ny, Nz = grid.N
    V = U[:, :3].reshape(Nz + 1, Ny + 1, Nx + 1, 3)
    hx, hy, hz = grid.h

    def face_integral(F, da, db):
        # exact integral of a bilinear field over a face grid of cells
        return da * db * 0.25 * (F[:-1, :-1] + F[1:, :-1] + F[:-1, 1:] + F[1:, 1:]).sum()

    flux = (face_integral(V[:, :, -1, 0], hz, hy) - face_integral(V[:, :, 0, 0], hz, hy)
            + face_integral(V[:, -1, :, 1], hz, hx) - face_integral(V[:, 0, :, 1], hz, hx)
            + face_integral(V[-1, :, :, 2], hy, hx) - face_integral(V[0, :, :, 2], hy, hx))
    assert R[:, 3].sum() == pytest.approx(flux, rel=1e-12, abs=1e-13)


def test_constant_state_has_no_interior_residual(oracle):
    core = oracle.core
    grid = core.Grid(4)
    n = grid.n_nodes
    U = np.tile([0.3, -0.7, 1.1, 2.5], (n, 1))
    A = np.zeros((n, 4))
    A[:, 3] = 1.0
    R = core.residual(grid, dict(rho=1.0, mu=0.01, dt=1e-3), U, A)
    X = grid.node_coords()
    interior = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    assert np.abs(R[interior]).max() < 1e-14
    assert np.abs(R[~interior, :3]).max() > 1e-3   # boundary pressure traction


@pytest.mark.parametrize("has_s", [False, True])
def test_jacobian_matches_central_differences(oracle, has_s):
    core = oracle.core
    rng = np.random.default_rng(3)
    grid = core.Grid((3, 4, 2), h=(0.3, 0.2, 0.4))
    n = grid.n_nodes
    U, A, f = rng.normal(size=(n, 4)), rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    A[:, 3] = rng.uniform(1.0, 3.0, n)
    x = rng.normal(size=(n, 4))
    c_a, c_v = 0.8, 0.05
    phys = dict(rho=1.2, mu=0.03, dt=0.02, has_s=has_s)
    Jx = core.jacobian_apply(grid, phys, U, A, x, c_a, c_v, f=f)
    dU = np.concatenate([c_v * x[:, :3], x[:, 3:]], axis=1)
    dA = np.concatenate([c_a * x[:, :3], np.zeros((n, 1))], axis=1)
    errs = []
    for eps in (1e-1, 1e-2, 1e-3):
        Rp = core.residual(grid, phys, U + eps * dU, A + eps * dA, f=f)
        Rm = core.residual(grid, phys, U - eps * dU, A - eps * dA, f=f)
        errs.append(np.linalg.norm((Rp - Rm) / (2 * eps) - Jx) / np.linalg.norm(Jx))
    assert errs[2] < 1e-8
    assert errs[0] > 1e-7   # the residual is genuinely nonlinear here
    assert 70.0 < errs[0] / errs[1] < 130.0   # second order: 100x per decade of eps


def test_element_jacobian_matches_apply(oracle):
    core = oracle.core
    from oracle import newton
    rng = np.random.default_rng(4)
    grid = core.Grid(2)
    n = grid.n_nodes
    U, A = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    phys = dict(rho=1.0, mu=0.1, dt=0.01)
    J = newton.assemble(grid, phys, U, A, 0.7, 0.02)
    x = rng.normal(size=(n, 4))
    Jx = core.jacobian_apply(grid, phys, U, A, x, 0.7, 0.02)
    assert np.abs(J @ x.ravel() - Jx.ravel()).max() < 1e-12 * np.abs(Jx).max()


def test_pspg_pressure_block_positive(oracle):
    """dR^c/dP = int grad q . (tau_M/rho) grad p: symmetric PSD, constants in its
    null space (the PSPG sign of the VMS form)."""
    core = oracle.core
    from oracle import newton
    rng = np.random.default_rng(8)
    grid = core.Grid(3)
    n = grid.n_nodes
    U, A = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    A[:, 3] = 1.0
    J = newton.assemble(grid, dict(rho=1.0, mu=0.01, dt=1e-2), U, A, 0.8, 0.01).toarray()
    Jpp = J[3::4, 3::4]
    assert np.abs(Jpp - Jpp.T).max() < 1e-14 * np.abs(Jpp).max()
    ev = np.linalg.eigvalsh(0.5 * (Jpp + Jpp.T))
    assert ev[0] > -1e-14 * ev[-1] and abs(ev[0]) < 1e-12 * ev[-1] and ev[1] > 1e-6 * ev[-1]
    assert np.abs(Jpp @ np.ones(n)).max() < 1e-14 * np.abs(Jpp).max()


# ---------------------------------------------------------------- manufactured
def _mms_exact(X, mu):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    pi = math.pi
    v = np.stack([pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z),
                  -pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z),
                  np.zeros_like(x)], axis=1)
    gv = np.zeros((len(x), 3, 3))
    gv[:, 0, 0] = pi * pi * np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * z)
    gv[:, 0, 1] = -pi * pi * np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
    gv[:, 0, 2] = pi * pi * np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * z)
    gv[:, 1, 0] = pi * pi * np.sin(pi * x) * np.sin(pi * y) * np.sin(pi * z)
    gv[:, 1, 1] = -pi * pi * np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * z)
    gv[:, 1, 2] = -pi * pi * np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * z)
    p = np.cos(pi * x) * np.cos(pi * y) * np.cos(pi * z)
    gp = -pi * np.stack([np.sin(pi * x) * np.cos(pi * y) * np.cos(pi * z),
                         np.cos(pi * x) * np.sin(pi * y) * np.cos(pi * z),
                         np.cos(pi * x) * np.cos(pi * y) * np.sin(pi * z)], axis=1)
    lap_v = -3.0 * pi * pi * v
    f = np.einsum("qj,qij->qi", v, gv) + gp - mu * lap_v
    return v, gv, p, f


def _mms_errors(grid, Uh, mu):
    P, W = wf.gauss_rule(3)
    Nq, dNxi = wf.q1_basis(P)
    h = np.asarray(grid.h)
    dN = dNxi * (2.0 / h)[None, None, :]
    detJ = np.prod(h) / 8.0
    ev2 = eg2 = 0.0
    pdiff, pw = [], []
    for e in range(grid.n_elems):
        ln = local_nodes(grid, e)
        N0 = grid.N
        ex, ey, ez = e % N0[0], (e // N0[0]) % N0[1], e // (N0[0] * N0[1])
        X = (np.array([ex, ey, ez]) + (P + 1) / 2) * h
        v, gv, p, _ = _mms_exact(X, mu)
        vh = Nq @ Uh[ln, :3]
        gvh = np.einsum("qaj,ai->qij", dN, Uh[ln, :3])
        ph = Nq @ Uh[ln, 3]
        ev2 += detJ * np.sum(W * np.sum((vh - v) ** 2, axis=1))
        eg2 += detJ * np.sum(W * np.sum((gvh - gv) ** 2, axis=(1, 2)))
        pdiff.append(ph - p)
        pw.append(detJ * W)
    pdiff, pw = np.concatenate(pdiff), np.concatenate(pw)
    pdiff -= np.sum(pw * pdiff) / np.sum(pw)
    return math.sqrt(ev2), math.sqrt(eg2), math.sqrt(np.sum(pw * pdiff ** 2))


def _mms_solve(oracle, N, mu=1.0):
    import scipy.sparse.linalg as spla
    from oracle import newton
    core = oracle.core
    grid = core.Grid(N)
    X = grid.node_coords()
    v, _, p, f = _mms_exact(X, mu)
    phys = dict(rho=1.0, mu=mu, dt=None)
    n = grid.n_nodes
    F = np.zeros((n, 4))
    F[:, :3] = f
    A = np.zeros((n, 4))
    A[:, 3] = 1.0
    bnd = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    mask = np.zeros((n, 4), dtype=bool)
    mask[bnd, :3] = True
    mask[0, 3] = True
    yD = np.zeros((n, 4))
    yD[:, :3] = v
    yD[:, 3] = p
    U = np.where(mask, yD, 0.0)
    hist = []
    for _ in range(12):
        R = core.residual(grid, phys, U, A, f=F)
        R[mask] = (U - yD)[mask]
        hist.append(np.linalg.norm(R))
        if hist[-1] < 1e-10:
            break
        J = newton.assemble(grid, phys, U, A, 0.0, 1.0, f=F).tolil()
        for r in np.flatnonzero(mask.ravel()):
            J.rows[r] = [int(r)]
            J.data[r] = [1.0]
        U = U + spla.spsolve(J.tocsc(), -R.ravel()).reshape(n, 4)
    return grid, U, hist


@pytest.mark.slow
def test_manufactured_solution_rates(oracle):
    """Steady Navier-Stokes MMS with Dirichlet velocity: the spatial rates must be
    near the optimal ones for Q1-Q1 VMS (the paper reports 2.0 / 1.5 / 1.5 for
    v L2 / p L2 / v H1 on its immersed benchmark, Sec. 4.1)."""
    errs = []
    for N in (4, 8, 16):
        grid, U, hist = _mms_solve(oracle, N)
        assert hist[-1] < 1e-10
        errs.append(_mms_errors(grid, U, 1.0))
    errs = np.array(errs)
    rates = np.log2(errs[:-1] / errs[1:])
    paper = GOLDEN["rates"]
    assert rates[-1, 0] > paper["v_L2"] - 0.2, rates   # v L2 (optimal 2)
    assert rates[-1, 1] > 0.9, rates                   # v H1 (optimal 1 for a smooth field)
    assert rates[-1, 2] > paper["p_L2"] - 0.1, rates   # p L2


def test_newton_converges_quadratically(oracle):
    grid, U, hist = _mms_solve(oracle, 4, mu=0.05)
    h = np.array(hist)
    assert h[-1] < 1e-10
    # quadratic: log-ratio of successive reductions approaches 2
    k = np.flatnonzero(h > 1e-9)
    r = np.log(h[k[-1] + 1] / h[k[-1]]) / np.log(h[k[-1]] / h[k[-1] - 1])
    assert r > 1.6, h
