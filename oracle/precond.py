"""Schur-complement block preconditioner of the Newton step: the pressure
operator, its grid hierarchy and one multigrid V-cycle, plain and assembled.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.4 solves the reduced system with block preconditioners built from its
sub-matrices.  Write the linearised fluid system per node block as

    [ A  B ] [dVdot]        A = dR^{f,m}/dVdot,  B = dR^{f,m}/dP,
    [ C  D ] [dP   ]        C = dR^{f,c}/dVdot,  D = dR^{f,c}/dP.

For the time steps of interest A is dominated by the mass term
alpha_m rho M, and B, C are the discrete gradient and (chain factor
c_v = alpha_f gamma dt times) divergence, so the pressure Schur complement
S = D - C A^{-1} B acts on smooth pressures like sigma K with K the Q1
stiffness ("Laplacian") matrix of the pressure space and
sigma = c_v / (alpha_m rho); on rough pressures the PSPG block D = tau_M/rho K
with tau_M ~ dt / sqrt(C_T) has the same size.  The preconditioner is

    z_v = blockdiag_3x3(A)^{-1} r_v,    z_p = S_hat^{-1} r_p,
    S_hat = sigma (K + kappa M),  kappa = (pi / (2 L))^2,

L the largest extent of the grid; the kappa M term (M the Q1 mass matrix) keeps
S_hat non-singular where only Neumann conditions bound the pressure.  On a
face of the box where the velocity is not prescribed (a traction-free outflow)
the true Schur complement behaves like a Dirichlet problem for the pressure
(its largest eigenvalues against sigma K live there and grow like 1/h), so the
nodes of such faces are eliminated from S_hat: their rows and columns are
dropped except the diagonal entry.  A face counts as such when more than half
of its nodes have all three velocity components free (``faces_from_mask``).
S_hat^{-1} is replaced by one V-cycle (the definitions below), a fixed linear
operator.

Definitions, all on a uniform grid with Q1 elements:
  K_e, M_e   element matrices int grad N_a . grad N_b and int N_a N_b, 2x2x2
             Gauss (exact for these integrands), assembled over all elements;
  A_l        K + kappa M on level l (kappa of the finest grid on every level);
  levels     the finest grid, then every other node (N_d -> N_d / 2) while all
             N_d are even and the grid has more than 125 nodes;
  P_l        trilinear interpolation from level l+1 to level l (the coarse Q1
             basis evaluated at the fine nodes), R_l = P_l^T;
  smoother   Chebyshev semi-iteration of degree nu on D^{-1} A_l (D its
             diagonal) over [hi / 4, hi], hi = 1.1 x the largest ratio of
             symbol to diagonal over the modes with theta_d in {0, pi};
  coarsest   a direct solve when it has at most 1000 nodes, otherwise a
             Chebyshev semi-iteration of degree 8 over [hi / 30, hi] from zero;
  V-cycle    x = smooth(nu, from 0); r = b - A x; x += P V(R r); x = smooth(nu, from x),
             with the restricted right-hand side zeroed on eliminated nodes.

Pins (tests/test_oracle_precond.py): K 1 = 0; u^T K u and u^T M u against the
integrals for trilinear u; Galerkin property P^T A_l P = A_{l+1}; exact
interpolation of trilinear fields by P; the smoother's error polynomial for a
diagonal operator equals the scaled Chebyshev polynomial; the spectrum bound
holds; the V-cycle contracts the error by a grid-independent factor.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

NU = 2                  # pre- and post-smoothing degree
DIRECT_MAX_NODES = 1000
COARSE_DEGREE = 8
MIN_COARSEN_NODES = 125


class Level:
    def __init__(self, N, h):
        self.N = tuple(int(v) for v in N)
        self.h = tuple(float(v) for v in h)
        self.n = (self.N[0] + 1) * (self.N[1] + 1) * (self.N[2] + 1)

    def face_nodes(self, faces):
        """Boolean [n]: nodes on the eliminated faces, faces = (x0, x1, y0, y1, z0, z1)."""
        ijk = np.indices((self.N[2] + 1, self.N[1] + 1, self.N[0] + 1)).reshape(3, -1)
        k, j, i = ijk
        on = np.zeros(self.n, dtype=bool)
        for d, idx in enumerate((i, j, k)):
            if faces[2 * d]:
                on |= idx == 0
            if faces[2 * d + 1]:
                on |= idx == self.N[d]
        return on


def faces_from_mask(N, mask):
    """Faces (x0, x1, y0, y1, z0, z1) on which more than half of the nodes
    inside the face (off its edges; all of its nodes if it has none inside)
    have all three velocity components free (mask [n, 4] of the Dirichlet rows)."""
    L = Level(N, (1.0, 1.0, 1.0))
    free = ~np.asarray(mask, dtype=bool)[:, :3].any(axis=1)
    k, j, i = np.indices((L.N[2] + 1, L.N[1] + 1, L.N[0] + 1)).reshape(3, -1)
    idx = (i, j, k)
    out = []
    for d in range(3):
        inner = np.ones(L.n, dtype=bool)
        for e in range(3):
            if e != d:
                inner &= (idx[e] > 0) & (idx[e] < L.N[e])
        for side in (0, L.N[d]):
            on = idx[d] == side
            sel = on & inner if np.any(on & inner) else on
            out.append(int(2 * np.count_nonzero(free & sel) > np.count_nonzero(sel)))
    return tuple(out)


def _element_matrices(h):
    """Q1 element stiffness and mass on an hx x hy x hz box (2x2x2 Gauss)."""
    g = 1.0 / math.sqrt(3.0)
    Ke = np.zeros((8, 8))
    Me = np.zeros((8, 8))
    detJ = h[0] * h[1] * h[2] / 8.0
    corners = [(a & 1, (a >> 1) & 1, (a >> 2) & 1) for a in range(8)]
    for q in range(8):
        xi = [(-g, g)[(q >> d) & 1] for d in range(3)]
        N = np.empty(8)
        G = np.empty((8, 3))
        for a, c in enumerate(corners):
            s = [2 * c[d] - 1 for d in range(3)]
            f = [0.5 * (1 + s[d] * xi[d]) for d in range(3)]
            N[a] = f[0] * f[1] * f[2]
            for d in range(3):
                df = 0.5 * s[d] * (2.0 / h[d])
                G[a, d] = df * np.prod([f[e] for e in range(3) if e != d])
        Ke += detJ * G @ G.T
        Me += detJ * np.outer(N, N)
    return Ke, Me


def _connectivity(N):
    nx, ny = N[0] + 1, N[1] + 1
    conn = []
    for ez in range(N[2]):
        for ey in range(N[1]):
            for ex in range(N[0]):
                n0 = ex + nx * (ey + ny * ez)
                conn.append([n0 + (a & 1) + nx * ((a >> 1) & 1) + nx * ny * ((a >> 2) & 1)
                             for a in range(8)])
    return np.array(conn, dtype=np.int64)


def assemble(level: Level, kappa: float = 0.0, faces=(0,) * 6):
    """(K + kappa M) with the nodes of `faces` eliminated (rows and columns
    dropped, diagonal kept), K and M of a level as CSR matrices."""
    Ke, Me = _element_matrices(level.h)
    conn = _connectivity(level.N)
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    E = conn.shape[0]
    K = sp.csr_matrix((np.tile(Ke.ravel(), E), (rows, cols)), shape=(level.n, level.n))
    M = sp.csr_matrix((np.tile(Me.ravel(), E), (rows, cols)), shape=(level.n, level.n))
    A = (K + kappa * M).tocsr()
    dirn = level.face_nodes(faces)
    if dirn.any():
        keep = sp.diags((~dirn).astype(float))
        A = (keep @ A @ keep + sp.diags(np.where(dirn, A.diagonal(), 0.0))).tocsr()
    return A, K, M


def kappa_of(N, h):
    L = max(N[d] * h[d] for d in range(3))
    return (math.pi / (2.0 * L)) ** 2


def hierarchy(N, h):
    levels = [Level(N, h)]
    while True:
        L = levels[-1]
        if L.n <= MIN_COARSEN_NODES or any(v % 2 for v in L.N):
            break
        levels.append(Level([v // 2 for v in L.N], [2 * v for v in L.h]))
    return levels


def prolongation(fine: Level, coarse: Level):
    """P[f, c] = coarse Q1 basis function c evaluated at fine node f."""
    rows, cols, vals = [], [], []
    nfx, nfy = fine.N[0] + 1, fine.N[1] + 1
    ncx, ncy = coarse.N[0] + 1, coarse.N[1] + 1

    def one_d(i):
        # fine index i -> list of (coarse index, weight)
        return [(i // 2, 1.0)] if i % 2 == 0 else [(i // 2, 0.5), (i // 2 + 1, 0.5)]

    for k in range(fine.N[2] + 1):
        for j in range(fine.N[1] + 1):
            for i in range(fine.N[0] + 1):
                f = i + nfx * (j + nfy * k)
                for ci, wi in one_d(i):
                    for cj, wj in one_d(j):
                        for ck, wk in one_d(k):
                            rows.append(f)
                            cols.append(ci + ncx * (cj + ncy * ck))
                            vals.append(wi * wj * wk)
    return sp.csr_matrix((vals, (rows, cols)), shape=(fine.n, coarse.n))


def spectrum_bound(h, kappa):
    """hi = 1.1 x max over theta in {0, pi}^3 of symbol(K + kappa M) / diagonal."""
    diag = sum((2.0 / h[d]) * np.prod([2.0 * h[e] / 3.0 for e in range(3) if e != d])
               for d in range(3)) + kappa * np.prod([2.0 * h[e] / 3.0 for e in range(3)])
    best = 0.0
    for s in range(8):
        pi_d = [(s >> d) & 1 for d in range(3)]
        k = [4.0 / h[d] if pi_d[d] else 0.0 for d in range(3)]
        m = [h[d] / 3.0 if pi_d[d] else h[d] for d in range(3)]
        sym = sum(k[d] * np.prod([m[e] for e in range(3) if e != d]) for d in range(3))
        sym += kappa * m[0] * m[1] * m[2]
        best = max(best, sym / diag)
    return 1.1 * best


def chebyshev(A, Dinv, b, x, degree, lo, hi):
    """Chebyshev semi-iteration for A x = b preconditioned by D^{-1} on the
    eigenvalue interval [lo, hi]: theta = (hi + lo)/2, delta = (hi - lo)/2,
    s1 = theta/delta; rho_0 = 1/s1, d_0 = D^{-1} r_0 / theta; then
    rho_k = 1/(2 s1 - rho_{k-1}), d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k/delta) D^{-1} r_k;
    x_{k+1} = x_k + d_k, r_{k+1} = b - A x_{k+1}."""
    theta, delta = 0.5 * (hi + lo), 0.5 * (hi - lo)
    s1 = theta / delta
    x = x.copy()
    r = b - A @ x
    d = Dinv * r / theta
    rho = 1.0 / s1
    for _ in range(degree - 1):
        x = x + d
        r = b - A @ x
        rho_new = 1.0 / (2.0 * s1 - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * (Dinv * r)
        rho = rho_new
    return x + d


class MultigridOracle:
    """The V-cycle of the module docstring, with assembled matrices."""

    def __init__(self, N, h=None, faces=(0,) * 6):
        N = (N, N, N) if np.isscalar(N) else tuple(N)
        h = tuple(1.0 / v for v in N) if h is None else tuple(h)
        self.kappa = kappa_of(N, h)
        self.faces = tuple(int(bool(f)) for f in faces)
        self.levels = hierarchy(N, h)
        self.A = [assemble(L, self.kappa, self.faces)[0] for L in self.levels]
        self.dirn = [L.face_nodes(self.faces) for L in self.levels]
        self.Dinv = [1.0 / A.diagonal() for A in self.A]
        self.hi = [spectrum_bound(L.h, self.kappa) for L in self.levels]
        self.P = [prolongation(self.levels[l], self.levels[l + 1])
                  for l in range(len(self.levels) - 1)]
        c = self.levels[-1]
        self.direct = c.n <= DIRECT_MAX_NODES
        if self.direct:
            self.coarse_lu = spla.splu(self.A[-1].tocsc())

    def smooth(self, l, b, x, degree=NU):
        return chebyshev(self.A[l], self.Dinv[l], b, x, degree, self.hi[l] / 4.0, self.hi[l])

    def coarse_solve(self, b):
        l = len(self.levels) - 1
        if self.direct:
            return self.coarse_lu.solve(b)
        return chebyshev(self.A[l], self.Dinv[l], b, np.zeros_like(b), COARSE_DEGREE,
                         self.hi[l] / 30.0, self.hi[l])

    def vcycle(self, b, l=0):
        if l == len(self.levels) - 1:
            return self.coarse_solve(b)
        x = self.smooth(l, b, np.zeros_like(b))
        r = b - self.A[l] @ x
        bc = self.P[l].T @ r
        bc[self.dirn[l + 1]] = 0.0
        x = x + self.P[l] @ self.vcycle(bc, l + 1)
        return self.smooth(l, b, x)


def sigma_of(rho, dt, rho_inf=0.5):
    """sigma = c_v / (alpha_m rho) of the generalized-alpha scheme."""
    from . import timeint
    am, af, gm = timeint.alphas(rho_inf)
    return af * gm * dt / (am * rho)


def mapped_pressure_operator(N, X, kappa=None, eliminated=None):
    """K + kappa M of the Q1 pressure space of a structured grid whose node
    (i, j, k) (number i + (Nx+1)(j + (Ny+1)k)) sits at X[node] (a trilinear
    map per element), as a scipy CSR matrix: the pressure Schur
    approximation sigma (K + kappa M) assembled on a mapped grid (Sec. 2.4; the module
    docstring's operator with the true geometry in place of the nominal box).
    Per element and Gauss point xi in {-1/sqrt3, 1/sqrt3}^3 (weight 1):
    J = sum_a x_a (grad_xi N_a)^T, grad N_a = J^-T grad_xi N_a,
    K_ab += |det J| grad N_a . grad N_b, M_ab += |det J| N_a N_b.  kappa
    defaults to (pi / (2 L))^2, L the largest extent of the nodes' bounding
    box.  Nodes flagged in `eliminated` keep only their diagonal entry.
    """
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    if kappa is None:
        L = float(np.max(X.max(axis=0) - X.min(axis=0)))
        kappa = (math.pi / (2.0 * L)) ** 2
    conn = _connectivity(N)
    g = 1.0 / math.sqrt(3.0)
    s = np.array([[2 * ((a >> d) & 1) - 1 for d in range(3)] for a in range(8)], dtype=float)
    xe = X[conn]                                   # [E, 8, 3]
    Ae = np.zeros((conn.shape[0], 8, 8))
    for q in range(8):
        xi = np.array([(-g, g)[(q >> d) & 1] for d in range(3)])
        f = 0.5 * (1.0 + s * xi[None, :])          # [8, 3] 1D factors
        Nq = f.prod(axis=1)                        # [8]
        dN = np.empty((8, 3))                      # d N_a / d xi_d
        for d in range(3):
            dN[:, d] = 0.5 * s[:, d] * np.prod(np.delete(f, d, axis=1), axis=1)
        J = np.einsum("eai,ad->eid", xe, dN)       # J[e, i, d] = dx_i / dxi_d
        Jinv = np.linalg.inv(J)                    # [e, d, i]
        G = np.einsum("ad,edi->eai", dN, Jinv)     # grad N_a
        w = np.abs(np.linalg.det(J))[:, None, None]
        Ae += w * (np.einsum("eai,ebi->eab", G, G) + kappa * np.outer(Nq, Nq)[None])
    rows = np.repeat(conn, 8, axis=1).ravel()
    cols = np.tile(conn, (1, 8)).ravel()
    A = sp.csr_matrix((Ae.ravel(), (rows, cols)), shape=(n, n))
    if eliminated is not None:
        el = np.asarray(eliminated, dtype=bool)
        A = A.tocoo()
        keep = (A.row == A.col) | ~(el[A.row] | el[A.col])
        A = sp.csr_matrix((A.data[keep], (A.row[keep], A.col[keep])), shape=A.shape)
    return A
