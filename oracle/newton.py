"""Newton step on the reduced FSI system of Sec. 2.4 with exact (direct) solves.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The reduced system of Sec. 2.4 couples the fluid residual R^f with the solid
through the FSI constraint matrix C:

    [ dR^{f,m}/dVdot + C dR^s/dUddot C^T ,  dR^{f,m}/dP ] [dVdot]     [R^{f,m} + C R^s]
    [ dR^{f,c}/dVdot                     ,  dR^{f,c}/dP ] [dP   ] = - [R^{f,c}         ]

and the solid acceleration follows as C^T dVdot.  The paper's solid residual
needs FEBio's constitutive code; this oracle (like the CUDA path) uses a
point-mass stand-in per solid point B located at the start of the step:

    r^s_B = (rho_s - rho_f) (a_B - g) + k dx_B,
    a_B   = (C^T Vdot_{n+1})_B,    dx_B = dt (C^T V_{n+1})_B,

spread with the point weights w_B, so that R^{f,m} += C W r^s and the solid
tangent block is C W ((rho_s - rho_f) + k gamma dt^2) C^T.

Dirichlet rows (mask != 0) are replaced by R = y - y_D with unit Jacobian rows.
Convergence: ||R(y_k)||_2 <= rtol * ||R(y_ref)||_2 over all rows, FP64.

Parity: pinned by quadratic convergence of the exact-solve iteration and by
the manufactured-solution convergence rates (tests/test_oracle_vms.py).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import core, timeint


def assemble(grid: core.Grid, phys, U, A, c_a, c_v, f=None, nthreads=0):
    """Assembled (4n x 4n) CSR Jacobian of the fluid residual."""
    Ke, conn = core.element_jacobian(grid, phys, U, A, c_a, c_v, f=f, nthreads=nthreads)
    E = Ke.shape[0]
    dof = (4 * conn[:, :, None] + np.arange(4)[None, None, :]).reshape(E, 32)
    rows = np.repeat(dof, 32, axis=1).ravel()
    cols = np.tile(dof, (1, 32)).ravel()
    n = 4 * grid.n_nodes
    return sp.csr_matrix((Ke.ravel(), (rows, cols)), shape=(n, n))


def coupling_matrix(grid: core.Grid, elem, xi):
    """C^T as a sparse (3m x 3n_nodes... velocity) operator on [n,4] vectors.

    Returns the sparse matrix Ct of shape (3m, 4n) with (C^T V)_B = Ct @ V.ravel().
    Built column by column from the oracle's interpolation on unit vectors is
    too slow, so the shape values come from ``core.shape``.
    """
    m = len(elem)
    rows, cols, vals = [], [], []
    N0 = grid.N
    for b in range(m):
        e = int(elem[b])
        if e < 0:
            continue
        ex, ey, ez = e % N0[0], (e // N0[0]) % N0[1], e // (N0[0] * N0[1])
        Nv, _ = core.shape(xi[b])
        for a in range(8):
            i, j, k = ex + (a & 1), ey + ((a >> 1) & 1), ez + ((a >> 2) & 1)
            nd = i + (N0[0] + 1) * (j + (N0[1] + 1) * k)
            for c in range(3):
                rows.append(3 * b + c)
                cols.append(4 * nd + c)
                vals.append(Nv[a])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * m, 4 * grid.n_nodes))


def _is_tet(mesh):
    from . import tet
    return isinstance(mesh, tet.TetMesh)


def tet_coupling_matrix(mesh, elem, lam):
    """C^T on a tetrahedral mesh: (C^T V)_B = sum_a N_a(lam_B) V_a (velocity)."""
    m = len(elem)
    rows, cols, vals = [], [], []
    for b in range(m):
        e = int(elem[b])
        if e < 0:
            continue
        l1, l2, l3 = lam[b]
        Nv = (1.0 - l1 - l2 - l3, l1, l2, l3)
        for a in range(4):
            nd = int(mesh.tets[e, a])
            for c in range(3):
                rows.append(3 * b + c)
                cols.append(4 * nd + c)
                vals.append(Nv[a])
    return sp.csr_matrix((vals, (rows, cols)), shape=(3 * m, 4 * mesh.n_nodes))


# the operators of the step on either mesh kind: the structured grid (core)
# or a tetrahedral mesh (tet)
def _residual(mesh, phys, U, A, f):
    if _is_tet(mesh):
        from . import tet
        return tet.residual(mesh, phys, U, A, f=f)
    return core.residual(mesh, phys, U, A, f=f)


def _assemble(mesh, phys, U, A, c_a, c_v, f):
    if _is_tet(mesh):
        from . import tet
        return tet.assemble(mesh, tet.element_jacobian(mesh, phys, U, A, c_a, c_v, f=f))
    return assemble(mesh, phys, U, A, c_a, c_v, f=f)


def _interp(mesh, elem, xi, U):
    if _is_tet(mesh):
        from . import tet
        return tet.interp(mesh, elem, xi, U)
    return core.interp(mesh, elem, xi, U)


def _spread(mesh, elem, xi, lam, w=None, F=None, accumulate=False):
    if _is_tet(mesh):
        from . import tet
        return tet.spread(mesh, elem, xi, lam, w=w, F=F, accumulate=accumulate)
    return core.spread(mesh, elem, xi, lam, w=w, F=F, accumulate=accumulate)


def _coupling(mesh, elem, xi):
    return tet_coupling_matrix(mesh, elem, xi) if _is_tet(mesh) else coupling_matrix(mesh, elem, xi)


def _locate(mesh, X):
    if _is_tet(mesh):
        from . import tet
        return tet.locate(mesh, X)
    return core.locate(mesh, X)


class Problem:
    """One implicit step: unknown y = [Vdot_{n+1} | P_{n+1}] per node, on a
    structured grid (core.Grid) or a tetrahedral mesh (tet.TetMesh)."""

    def __init__(self, grid, phys, Vn, An, f=None, s=None, mask=None, yD=None,
                 points=None, solid=None, body=None):
        self.grid, self.phys = grid, phys
        self.Vn, self.An, self.f, self.s = Vn, An, f, s
        self.mask = None if mask is None else np.asarray(mask, dtype=bool)
        self.yD = yD
        self.dt, self.rho_inf = phys["dt"], phys["rho_inf"]
        self.c_a, self.c_v = timeint.chain_factors(self.rho_inf, self.dt)
        self.points = points  # (elem, xi, w) or None
        self.solid = solid or {}
        # hyperelastic immersed solid (oracle/solid.py) instead of the point-mass
        # stand-in: dict(mesh, u, v, a (history at the solid nodes), mat, g);
        # its nodes, located at X + u_n, are the coupling points
        self.body = body
        if body is not None:
            x_n = body["mesh"].X + body["u"]
            e, xi, nout = _locate(grid, x_n)
            assert nout == 0, "solid nodes must lie inside the fluid grid"
            self.body_points = (e, xi)

    def body_residual(self, a_next):
        from . import solid as so
        b = self.body
        u_af, v_af, a_am, _, _ = so.kinematics(b["u"], b["v"], b["a"], a_next, self.dt,
                                               self.rho_inf)
        return so.residual(b["mesh"], u_af, v_af, a_am, b["u"], b["mat"], self.phys["mu"],
                           b.get("g", (0.0, 0.0, 0.0)))

    def body_tangent(self, a_next):
        """Dense dR^s/duddot_{n+1} [3 ns, 3 ns] (unit-vector applications)."""
        from . import solid as so
        b = self.body
        u_af, _, _, _, _ = so.kinematics(b["u"], b["v"], b["a"], a_next, self.dt, self.rho_inf)
        ca, cu, cv = so.chain(self.dt, self.rho_inf)
        ns = b["mesh"].ns
        K = np.zeros((3 * ns, 3 * ns))
        for col in range(3 * ns):
            x = np.zeros((ns, 3))
            x[col // 3, col % 3] = 1.0
            K[:, col] = so.tangent_apply(b["mesh"], u_af, b["u"], x, b["mat"], self.phys["mu"],
                                         ca, cu, cv).ravel()
        return K

    def stage(self, y):
        return timeint.stage(y, self.Vn, self.An, self.dt, self.rho_inf, s=self.s)

    def residual(self, y):
        U, A = self.stage(y)
        R = _residual(self.grid, self.phys, U, A, self.f)
        if self.points is not None:
            elem, xi, w = self.points
            drho = self.solid.get("drho", 0.5)
            k = self.solid.get("k", 0.0)
            gvec = np.asarray(self.solid.get("g", (0.0, 0.0, 0.0)))
            a = _interp(self.grid, elem, xi, y)
            V1 = np.zeros_like(y)
            V1[:, :3] = timeint.velocity_next(y, self.Vn, self.An, self.dt, self.rho_inf)
            dx = self.dt * _interp(self.grid, elem, xi, V1)
            rs = drho * (a - gvec[None, :]) + k * dx
            R = _spread(self.grid, elem, xi, rs, w=w, F=R, accumulate=True)
        if self.body is not None:
            elem, xi = self.body_points
            a_next = _interp(self.grid, elem, xi, y)             # uddot_{n+1} = C^T Vdot_{n+1}
            R = _spread(self.grid, elem, xi, self.body_residual(a_next), F=R, accumulate=True)
        if self.mask is not None:
            R = R.copy()
            R[self.mask] = (y - self.yD)[self.mask]
        return R

    def jacobian(self, y):
        U, A = self.stage(y)
        J = _assemble(self.grid, self.phys, U, A, self.c_a, self.c_v, self.f)
        if self.points is not None:
            elem, xi, w = self.points
            drho = self.solid.get("drho", 0.5)
            k = self.solid.get("k", 0.0)
            _, _, gamma = timeint.alphas(self.rho_inf)
            Ct = _coupling(self.grid, elem, xi)
            wv = np.ones(len(elem)) if w is None else np.asarray(w)
            D = sp.diags(np.repeat(wv * (drho + k * gamma * self.dt ** 2), 3))
            J = J + (Ct.T @ D @ Ct)
        if self.body is not None:
            elem, xi = self.body_points
            Ct = _coupling(self.grid, elem, xi)
            a_next = _interp(self.grid, elem, xi, y)
            J = J + Ct.T @ sp.csr_matrix(self.body_tangent(a_next)) @ Ct
        if self.mask is not None:
            J = J.tolil()
            idx = np.flatnonzero(self.mask.ravel())
            for r in idx:
                J.rows[r] = [int(r)]
                J.data[r] = [1.0]
            J = J.tocsr()
        return J


def newton(problem: Problem, y0, rtol=1e-8, max_iter=20, ref_norm=None):
    """Exact Newton; returns (y, history of ||R||_2)."""
    y = np.array(y0, dtype=np.float64)
    R = problem.residual(y)
    r0 = np.linalg.norm(R) if ref_norm is None else ref_norm
    hist = [np.linalg.norm(R)]
    for _ in range(max_iter):
        if hist[-1] <= rtol * r0:
            break
        J = problem.jacobian(y)
        dy = spla.spsolve(J.tocsc(), -R.ravel()).reshape(y.shape)
        y = y + dy
        R = problem.residual(y)
        hist.append(np.linalg.norm(R))
    return y, hist
