"""Pins of the oracle on mapped (curvilinear) structured grids: the uniform grid
given as coordinates reproduces the uniform operators; the operators are
frame-invariant under rotations of a distorted grid; the Jacobian is the
derivative of the residual; the manufactured-solution rates survive a smooth
mapping; point location inverts the trilinear map."""
import math

import numpy as np
import pytest

import weakform_ref as wf

PHYS = dict(rho=1.0, mu=0.02, dt=1e-2, rho_inf=0.5, has_s=True)


def local_nodes(grid, e):
    N = grid.N
    ex, ey, ez = e % N[0], (e // N[0]) % N[1], e // (N[0] * N[1])
    return np.array([(ex + (a & 1)) + (N[0] + 1) * ((ey + ((a >> 1) & 1))
                                                    + (N[1] + 1) * (ez + ((a >> 2) & 1)))
                     for a in range(8)])


def bubble_map(X, delta):
    """Smooth map of the unit cube onto itself (identity on its faces)."""
    b = np.sin(2 * math.pi * X[:, 0]) * np.sin(2 * math.pi * X[:, 1]) * np.sin(2 * math.pi * X[:, 2])
    return X + delta * b[:, None] * np.array([1.0, -0.7, 0.4])[None, :]


def random_fields(n, seed):
    rng = np.random.default_rng(seed)
    U, A, x, f = (rng.uniform(-1, 1, (n, 4)) for _ in range(4))
    A[:, 3] = rng.uniform(1, 3, n)
    return U, A, x, f


def test_uniform_coordinates_reproduce_the_uniform_operators(oracle):
    core = oracle.core
    g0 = core.Grid((4, 3, 5), x0=(0.1, -0.2, 0.3), h=(0.2, 0.3, 0.15))
    g1 = core.Grid((4, 3, 5), coords=g0.node_coords())
    U, A, x, f = random_fields(g0.n_nodes, 0)
    c_a, c_v = oracle.timeint.chain_factors(0.5, PHYS["dt"])
    R0, R1 = core.residual(g0, PHYS, U, A, f=f), core.residual(g1, PHYS, U, A, f=f)
    J0 = core.jacobian_apply(g0, PHYS, U, A, x, c_a, c_v, f=f)
    J1 = core.jacobian_apply(g1, PHYS, U, A, x, c_a, c_v, f=f)
    assert np.linalg.norm(R1 - R0) <= 1e-13 * np.linalg.norm(R0)
    assert np.linalg.norm(J1 - J0) <= 1e-13 * np.linalg.norm(J0)


def test_operators_are_frame_invariant_on_a_distorted_grid(oracle):
    """Rotate and translate the grid and every vector field: the momentum rows
    rotate with it, the continuity rows do not change (G -> Q G Q^T)."""
    core = oracle.core
    rng = np.random.default_rng(1)
    base = core.Grid((4, 4, 3)).node_coords()
    X = base + 0.04 * rng.uniform(-1, 1, base.shape)           # non-affine hexahedra
    ang = 0.9
    Q = np.array([[math.cos(ang), -math.sin(ang), 0.0], [math.sin(ang), math.cos(ang), 0.0],
                  [0.0, 0.0, 1.0]]) @ np.array([[1, 0, 0], [0, math.cos(0.4), -math.sin(0.4)],
                                                [0, math.sin(0.4), math.cos(0.4)]])
    g = core.Grid((4, 4, 3), coords=X)
    gq = core.Grid((4, 4, 3), coords=X @ Q.T + np.array([2.0, -1.0, 0.5]))
    U, A, x, f = random_fields(g.n_nodes, 2)

    def rot(F):
        G = F.copy()
        G[:, :3] = F[:, :3] @ Q.T
        return G
    c_a, c_v = oracle.timeint.chain_factors(0.5, PHYS["dt"])
    R = core.residual(g, PHYS, U, A, f=f)
    Rq = core.residual(gq, PHYS, rot(U), rot(A), f=rot(f))
    assert np.linalg.norm(Rq - rot(R)) <= 1e-12 * np.linalg.norm(R)
    J = core.jacobian_apply(g, PHYS, U, A, x, c_a, c_v, f=f)
    Jq = core.jacobian_apply(gq, PHYS, rot(U), rot(A), rot(x), c_a, c_v, f=rot(f))
    assert np.linalg.norm(Jq - rot(J)) <= 1e-12 * np.linalg.norm(J)
    # a planted mistake: treating the distorted grid as axis-aligned breaks it
    gu = core.Grid((4, 4, 3))
    assert np.linalg.norm(core.residual(gu, PHYS, U, A, f=f) - R) > 1e-3 * np.linalg.norm(R)


def test_mapped_jacobian_is_the_residual_derivative(oracle):
    core = oracle.core
    X = bubble_map(core.Grid(4).node_coords(), 0.04)
    g = core.Grid(4, coords=X)
    U, A, x, f = random_fields(g.n_nodes, 3)
    c_a, c_v = 0.8, 1.3           # chain factors of order one: the form is strongly nonlinear
    Jx = core.jacobian_apply(g, PHYS, U, A, x, c_a, c_v, f=f)

    def R(t):
        Ut, At = U.copy(), A.copy()
        Ut[:, :3] += c_v * t * x[:, :3]
        Ut[:, 3] += t * x[:, 3]
        At[:, :3] += c_a * t * x[:, :3]
        return core.residual(g, PHYS, Ut, At, f=f)
    errs = [np.linalg.norm((R(e) - R(-e)) / (2 * e) - Jx) / np.linalg.norm(Jx)
            for e in (1e-2, 1e-3)]
    assert errs[1] < 1e-7 and errs[0] / errs[1] > 50


def _mms_exact(X, mu):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    pi = math.pi
    v = np.stack([pi * np.sin(pi * x) * np.cos(pi * y) * np.sin(pi * z),
                  -pi * np.cos(pi * x) * np.sin(pi * y) * np.sin(pi * z), np.zeros_like(x)], 1)
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
    f = np.einsum("qj,qij->qi", v, gv) + gp + mu * 3.0 * pi * pi * v
    return v, gv, p, f


def _mms_mapped(oracle, N, delta, mu=1.0):
    import scipy.sparse.linalg as spla
    from oracle import newton
    core = oracle.core
    X = bubble_map(core.Grid(N).node_coords(), delta)
    grid = core.Grid(N, coords=X)
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
    for _ in range(12):
        R = core.residual(grid, phys, U, A, f=F)
        R[mask] = (U - yD)[mask]
        if np.linalg.norm(R) < 1e-10:
            break
        J = newton.assemble(grid, phys, U, A, 0.0, 1.0, f=F).tolil()
        for r in np.flatnonzero(mask.ravel()):
            J.rows[r] = [int(r)]
            J.data[r] = [1.0]
        U = U + spla.spsolve(J.tocsc(), -R.ravel()).reshape(n, 4)
    # errors with a 3-point rule through the element maps
    P, W = wf.gauss_rule(3)
    Nq, dNxi = wf.q1_basis(P)
    ev2 = eg2 = 0.0
    pd, pw = [], []
    for e in range(grid.n_elems):
        ln = local_nodes(grid, e)
        xq = Nq @ X[ln]
        Jm = np.einsum("ai,qak->qik", X[ln], dNxi)
        det = np.linalg.det(Jm)
        dN = np.einsum("qak,qkj->qaj", dNxi, np.linalg.inv(Jm))
        ve, gve, pe, _ = _mms_exact(xq, mu)
        vh = Nq @ U[ln, :3]
        gvh = np.einsum("qaj,ai->qij", dN, U[ln, :3])
        ev2 += np.sum(W * det * np.sum((vh - ve) ** 2, axis=1))
        eg2 += np.sum(W * det * np.sum((gvh - gve) ** 2, axis=(1, 2)))
        pd.append(Nq @ U[ln, 3] - pe)
        pw.append(W * det)
    pd, pw = np.concatenate(pd), np.concatenate(pw)
    pd -= np.sum(pw * pd) / np.sum(pw)
    return math.sqrt(ev2), math.sqrt(eg2), math.sqrt(np.sum(pw * pd ** 2))


@pytest.mark.slow
def test_manufactured_solution_rates_on_a_mapped_grid(oracle):
    e8 = _mms_mapped(oracle, 8, 0.02)
    e16 = _mms_mapped(oracle, 16, 0.02)
    rates = [math.log2(a / b) for a, b in zip(e8, e16)]
    assert rates[0] > 1.8 and rates[1] > 0.9 and rates[2] > 1.4, rates


def test_mapped_location_inverts_the_trilinear_map(oracle):
    core = oracle.core
    rng = np.random.default_rng(4)
    N = (5, 4, 3)
    X = core.Grid(N).node_coords()
    X = X + 0.03 * rng.uniform(-1, 1, X.shape) * np.array([1 / 5, 1 / 4, 1 / 3])
    g = core.Grid(N, coords=X)
    # points mapped from random (element, xi) away from the faces
    m = 300
    e_true = rng.integers(0, g.n_elems, m)
    xi_true = rng.uniform(-0.95, 0.95, (m, 3))
    P = np.zeros((m, 3))
    for b in range(m):
        Nv, _ = core.shape(xi_true[b])
        P[b] = Nv @ X[local_nodes(g, e_true[b])]
    P = np.concatenate([P, [[5.0, 0.5, 0.5], [-0.2, 0.5, 0.5]]])
    e, xi, nout = core.locate(g, P)
    assert nout == 2 and np.all(e[-2:] == -1)
    assert np.array_equal(e[:m], e_true.astype(np.int32))
    assert np.abs(xi[:m] - xi_true).max() < 1e-12
    # the uniform grid as coordinates locates like the uniform formula
    gu = core.Grid(N)
    Q = rng.uniform(0.01, 0.99, (200, 3))
    e0, xi0, _ = core.locate(gu, Q)
    e1, xi1, _ = core.locate(core.Grid(N, coords=gu.node_coords()), Q)
    assert np.array_equal(e0, e1) and np.abs(xi0 - xi1).max() < 1e-13


def test_mapped_location_on_strongly_distorted_grid(oracle):
    """Nodes moved by up to 0.2 h per axis: the brute-force search passes
    through many far elements whose Newton iteration wanders without settling;
    only a settled root inside the cube counts, so every point lands in the
    element it was mapped from."""
    core = oracle.core
    rng = np.random.default_rng(3)
    N = (7, 6, 5)
    X = core.Grid(N).node_coords()
    d = 0.2 * rng.uniform(-1, 1, X.shape) * (1.0 / np.array(N))[None, :]
    d[np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)] = 0.0
    X = X + d
    g = core.Grid(N, coords=X)
    m = 800
    rng = np.random.default_rng(4)
    e_true = rng.integers(0, g.n_elems, m)
    xi_true = rng.uniform(-0.95, 0.95, (m, 3))
    P = np.array([core.shape(xi_true[b])[0] @ X[local_nodes(g, e_true[b])] for b in range(m)])
    e, xi, nout = core.locate(g, P)
    assert nout == 0 and np.array_equal(e, e_true.astype(np.int32))
    assert np.abs(xi - xi_true).max() < 1e-12
