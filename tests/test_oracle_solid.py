"""Pins of the immersed-solid oracle (oracle/solid.py, Sec. 2.2)."""
import math

import numpy as np
import pytest

from oracle import solid as so

MU, LAM = 2.0, 5.0


def distorted_box(n=(3, 2, 2), seed=0, amp=0.05):
    m = so.box_mesh(n, (0.0, 0.0, 0.0), (1.5, 1.0, 0.8))
    rng = np.random.default_rng(seed)
    m.X = m.X + amp * rng.uniform(-1, 1, m.X.shape)    # general (non-affine) hexahedra
    return m


def rotation(axis, angle):
    axis = np.asarray(axis, float) / np.linalg.norm(axis)
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + math.sin(angle) * K + (1 - math.cos(angle)) * K @ K


def test_shape_functions_partition_of_unity_and_gauss_volume():
    for q in range(8):
        N, dN = so.shape(so.GAUSS[q])
        assert N.sum() == pytest.approx(1.0) and np.abs(dN.sum(axis=0)).max() < 1e-15
    m = so.box_mesh((2, 3, 1), (0, 0, 0), (2.0, 1.5, 0.5))
    assert m.volume() == pytest.approx(1.5)


def test_reference_state_and_rigid_rotations_are_stress_free():
    m = distorted_box()
    assert np.abs(so.internal_force(m, np.zeros((m.ns, 3)), MU, LAM)).max() < 1e-14
    R = rotation((1, 2, 0.5), 0.7)
    u = m.X @ R.T - m.X + np.array([0.3, -0.2, 0.1])
    assert np.abs(so.internal_force(m, u, MU, LAM)).max() < 1e-12
    # a rigid velocity of the current configuration (rotation rate +
    # translation, v = W x + c) has no viscous stress
    W = np.array([[0, -0.4, 0.2], [0.4, 0, -0.1], [-0.2, 0.1, 0]])
    v = (m.X + u) @ W.T + np.array([1.0, 2.0, 3.0])
    assert np.abs(so.viscous(m, u, v, 0.7)).max() < 1e-12


def test_patch_test_homogeneous_deformation():
    """F0 everywhere: interior nodes are in equilibrium, the sum of all nodal
    forces vanishes, and each face carries its traction P N |face|."""
    m = so.box_mesh((3, 3, 3), (0, 0, 0), (1.0, 1.0, 1.0))
    F0 = np.array([[1.1, 0.05, 0.0], [0.02, 0.95, 0.03], [0.0, -0.04, 1.02]])
    u = m.X @ F0.T - m.X
    f = so.internal_force(m, u, MU, LAM)
    P = so.neo_hookean_P(F0, MU, LAM)
    inner = np.all((m.X > 1e-12) & (m.X < 1 - 1e-12), axis=1)
    assert np.abs(f[inner]).max() < 1e-13
    assert np.abs(f.sum(axis=0)).max() < 1e-13
    top = (m.X[:, 0] > 1 - 1e-12) & np.all((m.X[:, 1:] > 1e-12) & (m.X[:, 1:] < 1 - 1e-12), axis=1)
    # interior nodes of the face x = 1 carry traction P e_x times their tributary area (1/3)^2
    assert np.allclose(f[top], P[:, 0] / 9.0, rtol=1e-12)


def test_internal_force_is_the_energy_gradient():
    m = distorted_box(seed=1)
    rng = np.random.default_rng(2)
    u = 0.08 * rng.normal(size=(m.ns, 3))
    f = so.internal_force(m, u, MU, LAM)
    eps = 1e-6
    for a, i in [(0, 0), (3, 1), (7, 2), (m.ns - 1, 0), (5, 2)]:
        up, um = u.copy(), u.copy()
        up[a, i] += eps
        um[a, i] -= eps
        fd = (so.energy(m, up, MU, LAM) - so.energy(m, um, MU, LAM)) / (2 * eps)
        assert fd == pytest.approx(f[a, i], rel=1e-7, abs=1e-9)


def test_tangent_is_the_force_derivative():
    m = distorted_box(seed=3)
    rng = np.random.default_rng(4)
    u = 0.1 * rng.normal(size=(m.ns, 3))
    du = 0.1 * rng.normal(size=(m.ns, 3))
    K = so.internal_tangent_apply(m, u, du, MU, LAM)
    errs = []
    for eps in (1e-3, 1e-4):
        fd = (so.internal_force(m, u + eps * du, MU, LAM)
              - so.internal_force(m, u - eps * du, MU, LAM)) / (2 * eps)
        errs.append(np.linalg.norm(fd - K) / np.linalg.norm(K))
    assert errs[1] < 1e-7 and 80 < errs[0] / errs[1] < 120      # O(eps^2)


def test_small_strain_limit_is_linear_elasticity():
    m = distorted_box(seed=5)
    rng = np.random.default_rng(6)
    du = rng.normal(size=(m.ns, 3))
    t = 1e-7
    f = so.internal_force(m, t * du, MU, LAM) / t
    # linear elasticity written out: sigma = lam tr(eps) I + 2 mu eps
    ref = np.zeros_like(f)
    for e in range(m.es):
        ue = du[m.conn[e]]
        for N, gX, det0 in m.gauss_geometry(e):
            H = ue.T @ gX
            eps_ = 0.5 * (H + H.T)
            sig = LAM * np.trace(eps_) * np.eye(3) + 2 * MU * eps_
            ref[m.conn[e]] += det0 * gX @ sig
    assert np.linalg.norm(f - ref) / np.linalg.norm(ref) < 1e-5


def test_consistent_mass_and_viscous_shear():
    m = so.box_mesh((2, 4, 2), (0, 0, 0), (1.0, 2.0, 0.5))
    c = np.array([0.3, -1.0, 2.0])
    acc = np.tile(c, (m.ns, 1))
    mass = so.inertia(m, acc, 0.7, f=(0.0, 0.0, 1.0))
    assert np.allclose(mass.sum(axis=0), 0.7 * 1.0 * (c - [0, 0, 1.0]))
    # simple shear v = (g y, 0, 0) with the undeformed configuration: D_xy = g/2,
    # the face y = 2 carries the traction 2 mu D e_y = (mu g, 0, 0) over area 0.5
    g, mu_f = 0.8, 0.3
    v = np.zeros((m.ns, 3))
    v[:, 0] = g * m.X[:, 1]
    d = so.viscous(m, np.zeros((m.ns, 3)), v, mu_f)
    top = m.X[:, 1] > 2 - 1e-12
    assert d[top].sum(axis=0) == pytest.approx([mu_f * g * 0.5, 0.0, 0.0], abs=1e-13)
    assert np.abs(d.sum(axis=0)).max() < 1e-13


def test_generalized_alpha_kinematics():
    rng = np.random.default_rng(7)
    u, v, a = (rng.normal(size=(5, 3)) for _ in range(3))
    dt = 0.01
    u_af, v_af, a_am, u1, v1 = so.kinematics(u, v, a, a, dt)
    assert np.allclose(u1, u + dt * v + 0.5 * dt * dt * a)     # constant acceleration
    assert np.allclose(v1, v + dt * a)
    ca, cu, cv = so.chain(dt)
    # chain factors are the derivatives of the stage values w.r.t. uddot_{n+1}
    da = rng.normal(size=(5, 3))
    k2 = so.kinematics(u, v, a, a + da, dt)
    assert np.allclose(k2[0] - u_af, cu * da) and np.allclose(k2[1] - v_af, cv * da)
    assert np.allclose(k2[2] - a_am, ca * da)
    assert cu == pytest.approx((2 / 3) * 0.25 * (1 + 5 / 6 - 2 / 3) ** 2 * dt * dt)


def test_coupled_problem_with_the_hyperelastic_body():
    """The reduced system with a hyperelastic immersed block: the Jacobian is the
    central difference of the residual, and exact Newton converges quadratically."""
    from oracle import core, newton
    grid = core.Grid(6)
    n = grid.n_nodes
    rng = np.random.default_rng(11)
    body_mesh = so.box_mesh((2, 2, 1), (0.3, 0.35, 0.4), (0.65, 0.6, 0.55))
    ns = body_mesh.ns
    body = dict(mesh=body_mesh, u=0.02 * rng.normal(size=(ns, 3)),
                v=0.1 * rng.normal(size=(ns, 3)), a=rng.normal(size=(ns, 3)),
                mat=dict(rho_s=1.5, rho_f=1.0, mu=50.0, lam=200.0), g=(0.0, 0.0, -1.0))
    phys = dict(rho=1.0, mu=0.05, dt=0.2, rho_inf=0.5)
    Vn, An = 0.3 * rng.normal(size=(n, 4)), 0.3 * rng.normal(size=(n, 4))
    P = newton.Problem(grid, phys, Vn, An, body=body)
    y = 3.0 * rng.normal(size=(n, 4))    # large enough to strain the block nonlinearly
    J = P.jacobian(y)
    x = rng.normal(size=(n, 4))
    Jx = (J @ x.ravel()).reshape(n, 4)
    errs = []
    for eps in (1e-3, 1e-4):
        fd = (P.residual(y + eps * x) - P.residual(y - eps * x)) / (2 * eps)
        errs.append(np.linalg.norm(fd - Jx) / np.linalg.norm(Jx))
    assert errs[1] < 1e-8 and errs[0] / errs[1] > 30            # O(eps^2)
    y_s, hist = newton.newton(P, y, rtol=1e-12)
    assert hist[-1] <= 1e-12 * hist[0]
    assert hist[2] / hist[1] < 10 * (hist[1] / hist[0]) ** 2 + 1e-14  # quadratic
