"""Pins of the oracle's Q1 / location / interpolation / spreading functions.

Each test checks the oracle against something other than itself: exact
reproduction of trilinear fields (Q1 contains them), brute force over all
elements, numpy's stable argsort, and the exact adjointness of interpolation
(C^T, Eq. nodal_solid_velo) and spreading (C, Eq. fsi_constraint_matrix).
"""
import itertools

import numpy as np
import pytest

from paper_2601_08266_gb300 import inputs


def trilinear(X, c):
    x, y, z = X[:, 0], X[:, 1], X[:, 2]
    return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * y + c[5] * x * z
            + c[6] * y * z + c[7] * x * y * z)


def test_shape_kronecker_partition_of_unity(oracle):
    core = oracle.core
    for a in range(8):
        xi_a = np.array([2 * (a & 1) - 1, 2 * ((a >> 1) & 1) - 1, 2 * ((a >> 2) & 1) - 1.0])
        N, _ = core.shape(xi_a)
        assert np.array_equal(N, np.eye(8)[a])
    rng = np.random.default_rng(1)
    for _ in range(20):
        xi = rng.uniform(-1, 1, 3)
        N, dN = core.shape(xi)
        assert abs(N.sum() - 1.0) < 1e-15
        assert np.abs(dN.sum(axis=0)).max() < 1e-15
        # derivative by central differences of the shape values
        for k in range(3):
            e = np.zeros(3)
            e[k] = 1e-6
            Np, _ = core.shape(xi + e)
            Nm, _ = core.shape(xi - e)
            assert np.abs((Np - Nm) / 2e-6 - dN[:, k]).max() < 1e-9


@pytest.mark.parametrize("N,x0,h", [((4, 4, 4), (0, 0, 0), None),
                                    ((3, 5, 2), (-0.2, 0.1, 0.3), (0.3, 0.2, 0.45))])
def test_interp_reproduces_trilinear(oracle, N, x0, h):
    core = oracle.core
    g = core.Grid(N, x0=x0, h=h)
    rng = np.random.default_rng(7)
    c = rng.normal(size=(3, 8))
    nodes = g.node_coords()
    U = np.zeros((g.n_nodes, 4))
    for i in range(3):
        U[:, i] = trilinear(nodes, c[i])
    U[:, 3] = rng.normal(size=g.n_nodes)  # pressure slot must be ignored
    lo = np.asarray(g.x0)
    hi = lo + np.asarray(g.h) * np.asarray(g.N)
    X = lo + rng.uniform(0, 1, size=(500, 3)) * (hi - lo)
    elem, xi, nout = core.locate(g, X)
    assert nout == 0
    u = core.interp(g, elem, xi, U)
    for i in range(3):
        ref = trilinear(X, c[i])
        assert np.abs(u[:, i] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_locate_brute_force(oracle):
    core = oracle.core
    for N, h in [((4, 4, 4), None), ((3, 2, 5), (0.25, 0.5, 0.2))]:
        g = core.Grid(N, h=h)
        X = inputs.edge_points(g.N, seed=3, m_random=300)
        X = X * (np.asarray(g.h) * np.asarray(g.N))[None, :]
        elem, xi, nout = core.locate(g, X)
        hvec = np.asarray(g.h)
        n_out_ref = 0
        for b in range(len(X)):
            cands = []
            for ex, ey, ez in itertools.product(range(N[0]), range(N[1]), range(N[2])):
                lo = np.array([ex, ey, ez]) * hvec
                if np.all(X[b] >= lo) and np.all(X[b] <= lo + hvec):
                    cands.append(ex + N[0] * (ey + N[1] * ez))
            if not cands:
                n_out_ref += 1
                assert elem[b] == -1 and np.all(xi[b] == 0)
                continue
            assert elem[b] in cands
            # tie-break: floor rule with the upper face clamped (largest index
            # of a containing element along each axis, unless on the far face)
            e = elem[b]
            idx = np.array([e % N[0], (e // N[0]) % N[1], e // (N[0] * N[1])])
            t = X[b] / hvec
            want = np.minimum(np.floor(t).astype(int), np.asarray(N) - 1)
            assert np.array_equal(idx, want)
            assert np.all(np.abs(xi[b]) <= 1.0)
            back = (idx + (xi[b] + 1.0) / 2.0) * hvec
            assert np.abs(back - X[b]).max() < 1e-14
        assert nout == n_out_ref


def test_cell_hash_stable_counting_sort(oracle):
    core = oracle.core
    g = core.Grid(6)
    X = inputs.edge_points(g.N, seed=5, m_random=2000)
    elem, _, nout = core.locate(g, X)
    cs, perm = core.cell_hash(g, elem)
    inside = np.flatnonzero(elem >= 0)
    order = inside[np.argsort(elem[inside], kind="stable")]
    assert np.array_equal(perm[: len(inside)], order)
    assert np.array_equal(perm[len(inside):], np.flatnonzero(elem < 0))
    counts = np.bincount(elem[inside], minlength=g.n_elems)
    assert np.array_equal(np.diff(cs), counts)
    assert cs[0] == 0 and cs[-1] == len(inside) == len(X) - nout


@pytest.mark.parametrize("weighted", [False, True])
def test_spread_is_adjoint_of_interp(oracle, weighted):
    """<C^T V, lambda>_W = <V, C W lambda>: spreading is the transpose of
    interpolation (Eq. fsi_constraint_matrix vs Eq. nodal_solid_velo)."""
    core = oracle.core
    g = core.Grid((5, 4, 6), h=(0.2, 0.25, 1 / 6))
    rng = np.random.default_rng(11)
    X = inputs.ball_points(400, seed=2, radius=0.45)
    X = np.concatenate([X, inputs.edge_points(g.N, seed=4, m_random=10)])
    elem, xi, _ = core.locate(g, X)
    V = rng.normal(size=(g.n_nodes, 4))
    lam = rng.normal(size=(len(X), 3))
    w = rng.uniform(0.5, 2.0, size=len(X)) if weighted else None
    u = core.interp(g, elem, xi, V)
    F = core.spread(g, elem, xi, lam, w=w)
    wv = np.ones(len(X)) if w is None else w
    lhs = np.sum(wv[:, None] * u * lam)
    rhs = np.sum(V[:, :3] * F[:, :3])
    assert abs(lhs - rhs) <= 1e-13 * np.sum(np.abs(wv[:, None] * u * lam))
    # force conservation (partition of unity): sum_A F_A = sum_B w_B lambda_B
    inside = elem >= 0
    tot = (wv[inside, None] * lam[inside]).sum(axis=0)
    assert np.abs(F[:, :3].sum(axis=0) - tot).max() < 1e-12 * np.abs(lam).sum()
    # the pressure slot is never touched
    assert np.all(F[:, 3] == 0)


def test_spread_accumulate_and_single_point(oracle):
    core = oracle.core
    g = core.Grid(3)
    X = np.array([[0.4, 0.55, 0.9]])
    elem, xi, _ = core.locate(g, X)
    lam = np.array([[1.0, -2.0, 0.5]])
    F0 = np.full((g.n_nodes, 4), 3.0)
    F = core.spread(g, elem, xi, lam, F=F0, accumulate=True)
    Nv, _ = core.shape(xi[0])
    e = elem[0]
    ex, ey, ez = e % 3, (e // 3) % 3, e // 9
    expect = F0.copy()
    for a in range(8):
        nd = (ex + (a & 1)) + 4 * ((ey + ((a >> 1) & 1)) + 4 * (ez + ((a >> 2) & 1)))
        expect[nd, :3] += Nv[a] * lam[0]
    assert np.abs(F - expect).max() < 1e-15
