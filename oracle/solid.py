"""Immersed hyperelastic solid of Sec. 2.2 on a Q1 hexahedral solid mesh, plain.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The solid weak form of Sec. 2.2 (Eq. solid_weak_form):

    R_s(w, udot) = int_{Omega^s_t} w . (rho_s - rho_f)(uddot - f)
                 + int_{Omega^s_t} grad w : sigma
                 - int_{Omega^s_t} 2 mu_f eps(w) : eps(v^f)          (- traction, none here)

with sigma = (2/J) F dpsi/dC F^T.  Discretised here on trilinear hexahedra with
2x2x2 Gauss quadrature in the reference configuration (nodes X_a, corner a =
ax + 2 ay + 4 az, N_a = prod_k (1 + s_k xi_k)/2, s_k = 2 a_k - 1), nodal
values of the displacement u, velocity v and acceleration uddot:

  inertia    m_a = sum_g N_a (rho_s - rho_f) (uddot(g) - f) det J0   (consistent mass)
  internal   f_a = sum_g P(F) grad_X N_a det J0,  int grad w : sigma dOmega_t
             written with the first Piola-Kirchhoff stress P = J sigma F^{-T}
  viscous    d_a = sum_g 2 mu_f D(g) grad_x N_a J det J0,  D = sym(L),
             L = sum_b v_b (x) grad_x N_b,  grad_x N = grad_X N F^{-1}

  R^s_a = m_a + f_a - d_a.

Readings (the paper fixes none of these):
  material   compressible neo-Hookean psi = mu/2 (I1 - 3) - mu ln J + lam/2 (ln J)^2,
             P = mu (F - F^{-T}) + lam ln J F^{-T};
  viscous    the artificial fluid's velocity inside the solid is the solid's own
             velocity field (the constraint makes them equal at the solid nodes),
             and the configuration of the viscous term is the one at the start of
             the step (frozen like the constraint matrix C), so the term is linear
             in v;
  time       generalized-alpha with Newmark beta = (1 + alpha_m - alpha_f)^2 / 4:
             given uddot_{n+1}, v_{n+1} = v_n + dt ((1-gamma) a_n + gamma a_{n+1}),
             u_{n+1} = u_n + dt v_n + dt^2 ((1/2 - beta) a_n + beta a_{n+1}); the
             residual is taken at uddot_{n+alpha_m}, v_{n+alpha_f}, u_{n+alpha_f}
             (chain factors alpha_m, alpha_f gamma dt, alpha_f beta dt^2);
  coupling   the solid nodes are the Lagrange multiplier points (delta basis,
             Sec. 2.3): uddot_{n+1} = C^T Vdot_{n+1}, R^{f,m} += C R^s and the
             solid block of the reduced Jacobian is C dR^s/dUddot C^T.

Pins (tests/test_oracle_solid.py): zero force in the reference state and under
rigid rotations; the patch test (homogeneous deformation: interior nodal forces
vanish, boundary forces are the traction P N of the faces); internal force =
dW/du by central differences of the strain energy; the tangent = central
differences of the internal force; the small-strain limit against linear
elasticity; the consistent mass against the solid volume; the viscous term
against a hand-computed shear.
"""
from __future__ import annotations

import math

import numpy as np

G = 1.0 / math.sqrt(3.0)
CORNERS = np.array([[(a >> k) & 1 for k in range(3)] for a in range(8)], dtype=float)
SIGNS = 2.0 * CORNERS - 1.0
GAUSS = np.array([[(-G, G)[(q >> k) & 1] for k in range(3)] for q in range(8)])


def shape(xi):
    """N [8], dN/dxi [8, 3] of the trilinear hexahedron at xi [3]."""
    f = 0.5 * (1.0 + SIGNS * xi[None, :])            # [8, 3]
    N = f.prod(axis=1)
    dN = np.empty((8, 3))
    for k in range(3):
        others = [d for d in range(3) if d != k]
        dN[:, k] = 0.5 * SIGNS[:, k] * f[:, others[0]] * f[:, others[1]]
    return N, dN


def neo_hookean_P(F, mu, lam):
    J = np.linalg.det(F)
    Finv_T = np.linalg.inv(F).T
    return mu * (F - Finv_T) + lam * math.log(J) * Finv_T


def neo_hookean_dP(F, dF, mu, lam):
    """Directional derivative of P at F along dF."""
    J = np.linalg.det(F)
    Finv = np.linalg.inv(F)
    Finv_T = Finv.T
    return (mu * dF + (mu - lam * math.log(J)) * Finv_T @ dF.T @ Finv_T
            + lam * np.trace(Finv @ dF) * Finv_T)


def strain_energy(F, mu, lam):
    J = np.linalg.det(F)
    I1 = np.trace(F.T @ F)
    return 0.5 * mu * (I1 - 3.0) - mu * math.log(J) + 0.5 * lam * math.log(J) ** 2


class SolidMesh:
    """Reference nodes X [ns, 3], hex connectivity conn [es, 8] (corner order a)."""

    def __init__(self, X, conn):
        self.X = np.asarray(X, dtype=float)
        self.conn = np.asarray(conn, dtype=np.int64)
        self.ns, self.es = self.X.shape[0], self.conn.shape[0]

    def gauss_geometry(self, e):
        """Per Gauss point: N [8], grad_X N [8, 3], det J0."""
        Xe = self.X[self.conn[e]]
        out = []
        for q in range(8):
            N, dN = shape(GAUSS[q])
            J0 = Xe.T @ dN                          # J0[i, k] = sum_a X_ai dN_a/dxi_k
            det0 = np.linalg.det(J0)
            gX = dN @ np.linalg.inv(J0)             # grad_X N_a = J0^{-T} dN_a/dxi
            out.append((N, gX, det0))
        return out

    def volume(self):
        return sum(det0 for e in range(self.es) for (_, _, det0) in self.gauss_geometry(e))


def internal_force(mesh: SolidMesh, u, mu, lam):
    f = np.zeros((mesh.ns, 3))
    for e in range(mesh.es):
        ue = u[mesh.conn[e]]
        for N, gX, det0 in mesh.gauss_geometry(e):
            F = np.eye(3) + ue.T @ gX
            P = neo_hookean_P(F, mu, lam)
            f[mesh.conn[e]] += det0 * gX @ P.T      # f_ai += sum_j P_ij dN_a/dX_j
    return f


def energy(mesh: SolidMesh, u, mu, lam):
    W = 0.0
    for e in range(mesh.es):
        ue = u[mesh.conn[e]]
        for N, gX, det0 in mesh.gauss_geometry(e):
            W += det0 * strain_energy(np.eye(3) + ue.T @ gX, mu, lam)
    return W


def internal_tangent_apply(mesh: SolidMesh, u, du, mu, lam):
    df = np.zeros((mesh.ns, 3))
    for e in range(mesh.es):
        ue, due = u[mesh.conn[e]], du[mesh.conn[e]]
        for N, gX, det0 in mesh.gauss_geometry(e):
            F = np.eye(3) + ue.T @ gX
            dF = due.T @ gX
            df[mesh.conn[e]] += det0 * gX @ neo_hookean_dP(F, dF, mu, lam).T
    return df


def inertia(mesh: SolidMesh, a, drho, f=(0.0, 0.0, 0.0)):
    m = np.zeros((mesh.ns, 3))
    f = np.asarray(f, dtype=float)
    for e in range(mesh.es):
        ae = a[mesh.conn[e]]
        for N, gX, det0 in mesh.gauss_geometry(e):
            ag = N @ ae
            m[mesh.conn[e]] += det0 * drho * np.outer(N, ag - f)
    return m


def viscous(mesh: SolidMesh, u_cfg, v, mu_f):
    """d_a = sum_g 2 mu_f D grad_x N_a J det J0 on the configuration X + u_cfg."""
    d = np.zeros((mesh.ns, 3))
    for e in range(mesh.es):
        ue, ve = u_cfg[mesh.conn[e]], v[mesh.conn[e]]
        for N, gX, det0 in mesh.gauss_geometry(e):
            F = np.eye(3) + ue.T @ gX
            J = np.linalg.det(F)
            gx = gX @ np.linalg.inv(F)              # grad_x N_a (rows)
            L = ve.T @ gx                           # L_ij = sum_b v_bi dN_b/dx_j
            D = 0.5 * (L + L.T)
            d[mesh.conn[e]] += det0 * J * 2.0 * mu_f * gx @ D.T
    return d


def residual(mesh: SolidMesh, u_af, v_af, a_am, u_cfg, mat, mu_f, f=(0.0, 0.0, 0.0)):
    """R^s [ns, 3] = inertia + internal - viscous (mat = dict rho_s, rho_f, mu, lam)."""
    drho = mat["rho_s"] - mat["rho_f"]
    return (inertia(mesh, a_am, drho, f) + internal_force(mesh, u_af, mat["mu"], mat["lam"])
            - viscous(mesh, u_cfg, v_af, mu_f))


def tangent_apply(mesh: SolidMesh, u_af, u_cfg, x, mat, mu_f, c_a, c_u, c_v):
    """dR^s/duddot_{n+1} x with chain factors c_a = alpha_m (inertia),
    c_u = alpha_f beta dt^2 (internal force), c_v = alpha_f gamma dt (viscous)."""
    drho = mat["rho_s"] - mat["rho_f"]
    return (c_a * inertia(mesh, x, drho) + c_u * internal_tangent_apply(mesh, u_af, x, mat["mu"],
                                                                         mat["lam"])
            - c_v * viscous(mesh, u_cfg, x, mu_f))


def kinematics(u_n, v_n, a_n, a_next, dt, rho_inf=0.5):
    """(u_af, v_af, a_am, u_next, v_next) of generalized-alpha with Newmark beta."""
    from . import timeint
    am, af, gm = timeint.alphas(rho_inf)
    beta = 0.25 * (1.0 + am - af) ** 2
    v_next = v_n + dt * ((1.0 - gm) * a_n + gm * a_next)
    u_next = u_n + dt * v_n + dt * dt * ((0.5 - beta) * a_n + beta * a_next)
    return (u_n + af * (u_next - u_n), v_n + af * (v_next - v_n), a_n + am * (a_next - a_n),
            u_next, v_next)


def chain(dt, rho_inf=0.5):
    """(c_a, c_u, c_v) = (alpha_m, alpha_f beta dt^2, alpha_f gamma dt)."""
    from . import timeint
    am, af, gm = timeint.alphas(rho_inf)
    beta = 0.25 * (1.0 + am - af) ** 2
    return am, af * beta * dt * dt, af * gm * dt


def box_mesh(n, lo, hi):
    """Structured hex mesh of the box [lo, hi] with n = (nx, ny, nz) elements."""
    nx, ny, nz = n
    ax = [np.linspace(lo[d], hi[d], n[d] + 1) for d in range(3)]
    Z, Y, Xc = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    X = np.stack([Xc.ravel(), Y.ravel(), Z.ravel()], axis=1)
    conn = []
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                n0 = i + (nx + 1) * (j + (ny + 1) * k)
                conn.append([n0 + (a & 1) + (nx + 1) * ((a >> 1) & 1)
                             + (nx + 1) * (ny + 1) * ((a >> 2) & 1) for a in range(8)])
    return SolidMesh(X, np.array(conn))
