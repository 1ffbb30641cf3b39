"""Unstructured tetrahedral background meshes (linear P1-P1 tetrahedra, the
element family of the paper's valve fluid mesh, Sec. 4), plain.

TEST INFRASTRUCTURE ONLY (see the package docstring).

ctypes wrappers over the tetrahedral part of ``fsi_oracle.c``: the VMS
residual and its consistent Jacobian-vector product (the same weak form per
quadrature point as on hexahedra, Sec. 2.1 / Sec. 2.4, on the reference
tetrahedron with the symmetric 4-point rule of degree 2 and G = J^-T J^-1),
element Jacobians for direct Newton solves, brute-force point location by
barycentric coordinates (first element in element order whose coordinates are
all >= -1e-12), interpolation (Eq. nodal_solid_velo) and spreading
(Eq. fsi_constraint_matrix) with the barycentric shape functions.

Readings (the paper fixes none of them): the reference tetrahedron with unit
legs as the parent domain of G, C_I = 36 and C_T = 4 as on hexahedra, the
4-point rule (exact for the degree-2 Galerkin products of P1 fields).
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import core
from .core import _f64, _p, phys_array

_ready = False


def _lib():
    global _ready
    L = core.lib()
    if not _ready:
        d = ctypes.POINTER(ctypes.c_double)
        i32 = ctypes.POINTER(ctypes.c_int32)
        I64, C, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.or_tet_residual.argtypes = [I64, d, I64, i32, d, d, d, d, C, d, C]
        L.or_tet_jacobian_apply.argtypes = [I64, d, I64, i32, d, d, d, d, d, D, D, d, C]
        L.or_tet_element_jacobian.argtypes = [d, I64, i32, d, d, d, d, D, D, d, C]
        L.or_tet_barycentric.argtypes = [d, i32, d, d]
        L.or_tet_locate.argtypes = [d, I64, i32, I64, d, i32, d]
        L.or_tet_locate.restype = I64
        L.or_tet_interp.argtypes = [i32, I64, i32, d, d, d]
        L.or_tet_spread.argtypes = [I64, i32, I64, i32, d, d, d, d, C]
        _ready = True
    return L


class TetMesh:
    """Nodes X [n, 3] and tetrahedra tets [E, 4] (node numbers)."""

    def __init__(self, X, tets):
        self.X = _f64(X)
        self.tets = np.ascontiguousarray(tets, dtype=np.int32)
        self.n_nodes, self.n_elems = self.X.shape[0], self.tets.shape[0]
        assert self.X.shape == (self.n_nodes, 3) and self.tets.shape == (self.n_elems, 4)

    def volumes(self):
        e = self.X[self.tets[:, 1:]] - self.X[self.tets[:, :1]]
        return np.abs(np.linalg.det(np.transpose(e, (0, 2, 1)))) / 6.0


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def residual(mesh: TetMesh, phys, U, A, f=None, stab=True, nthreads=0):
    n = mesh.n_nodes
    U, A = _f64(U, (n, 4)), _f64(A, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    R = np.zeros((n, 4))
    _lib().or_tet_residual(n, _p(mesh.X), mesh.n_elems, _p(mesh.tets, ctypes.c_int32),
                           _p(phys_array(phys)), _p(U), _p(A), _p(f), 1 if stab else 0, _p(R),
                           int(nthreads))
    return R


def jacobian_apply(mesh: TetMesh, phys, U, A, x, c_a, c_v, f=None, nthreads=0):
    n = mesh.n_nodes
    U, A, x = _f64(U, (n, 4)), _f64(A, (n, 4)), _f64(x, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    Jx = np.zeros((n, 4))
    _lib().or_tet_jacobian_apply(n, _p(mesh.X), mesh.n_elems, _p(mesh.tets, ctypes.c_int32),
                                 _p(phys_array(phys)), _p(U), _p(A), _p(f), _p(x), float(c_a),
                                 float(c_v), _p(Jx), int(nthreads))
    return Jx


def element_jacobian(mesh: TetMesh, phys, U, A, c_a, c_v, f=None, nthreads=0):
    """Ke [E, 16, 16]: rows 4 a + c of the element residual, columns 4 b + d."""
    n = mesh.n_nodes
    U, A = _f64(U, (n, 4)), _f64(A, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    Ke = np.zeros((mesh.n_elems, 16, 16))
    _lib().or_tet_element_jacobian(_p(mesh.X), mesh.n_elems, _p(mesh.tets, ctypes.c_int32),
                                   _p(phys_array(phys)), _p(U), _p(A), _p(f), float(c_a),
                                   float(c_v), _p(Ke), int(nthreads))
    return Ke


def assemble(mesh: TetMesh, Ke):
    """Global sparse matrix [4n, 4n] of the element Jacobians."""
    import scipy.sparse as sp
    dof = (4 * mesh.tets[:, :, None] + np.arange(4)[None, None, :]).reshape(-1, 16)
    rows = np.repeat(dof, 16, axis=1).ravel()
    cols = np.tile(dof, (1, 16)).ravel()
    n4 = 4 * mesh.n_nodes
    return sp.csr_matrix((Ke.reshape(-1), (rows, cols)), shape=(n4, n4))


def barycentric(mesh: TetMesh, e, P):
    lam = np.zeros(4)
    _lib().or_tet_barycentric(_p(mesh.X), _p(mesh.tets[e], ctypes.c_int32),
                              _p(_f64(P, (3,))), _p(lam))
    return lam


def locate(mesh: TetMesh, P):
    P = _f64(P)
    m = P.shape[0]
    elem = np.empty(m, dtype=np.int32)
    lam = np.zeros((m, 3))
    nout = _lib().or_tet_locate(_p(mesh.X), mesh.n_elems, _p(mesh.tets, ctypes.c_int32), m,
                                _p(P), _p(elem, ctypes.c_int32), _p(lam))
    return elem, lam, int(nout)


def cell_hash(mesh: TetMesh, elem):
    """Element -> points CSR (stable counting sort), as on the grid."""
    E = mesh.n_elems
    m = len(elem)
    elem = _i32(elem)
    cs = np.zeros(E + 1, dtype=np.int32)
    perm = np.zeros(m, dtype=np.int32)
    Nc = (ctypes.c_int * 3)(E, 1, 1)
    core.lib().or_cell_hash(Nc, m, _p(elem, ctypes.c_int32), _p(cs, ctypes.c_int32),
                            _p(perm, ctypes.c_int32))
    return cs, perm


def interp(mesh: TetMesh, elem, lam, U):
    m = len(elem)
    u = np.zeros((m, 3))
    _lib().or_tet_interp(_p(mesh.tets, ctypes.c_int32), m, _p(_i32(elem), ctypes.c_int32),
                         _p(_f64(lam, (m, 3))), _p(_f64(U, (mesh.n_nodes, 4))), _p(u))
    return u


def spread(mesh: TetMesh, elem, lam, lamv, w=None, F=None, accumulate=False):
    m = len(elem)
    F = np.zeros((mesh.n_nodes, 4)) if F is None else _f64(F, (mesh.n_nodes, 4)).copy()
    _lib().or_tet_spread(mesh.n_nodes, _p(mesh.tets, ctypes.c_int32), m,
                         _p(_i32(elem), ctypes.c_int32), _p(_f64(lam, (m, 3))),
                         _p(_f64(lamv, (m, 3))), None if w is None else _p(_f64(w, (m,))),
                         _p(F), 1 if accumulate else 0)
    return F


def pressure_operator(mesh: TetMesh, kappa, eliminated=None):
    """K + kappa M of the P1 pressure space as a scipy CSR matrix [n, n]: the
    pressure Schur approximation sigma (K + kappa M) of the block
    preconditioner (Sec. 2.4 builds its block preconditioners from the
    sub-matrices of the reduced system; the stiffness-plus-mass form is the
    reading used on the structured grid too).  Per element, with the
    barycentric functions l_a(x) = c_a0 + c_a . x read off the inverse of
    [1 x_b] (rows b = corners): K_ab = V c_a . c_b, M_ab = V (1 + delta_ab) / 20,
    V = |det [1 x_b]| / 6.  Nodes flagged in `eliminated` keep only their
    diagonal entry (their rows and columns are dropped otherwise).
    """
    import scipy.sparse as sp
    E = mesh.n_elems
    M4 = np.ones((E, 4, 4))
    M4[:, :, 1:] = mesh.X[mesh.tets]
    C = np.linalg.inv(M4)               # column a: (c_a0, c_a)
    grad = np.transpose(C[:, 1:, :], (0, 2, 1))   # [E, a, 3]
    V = np.abs(np.linalg.det(M4)) / 6.0
    Ke = V[:, None, None] * np.einsum("eai,ebi->eab", grad, grad)
    Me = V[:, None, None] * (np.ones((4, 4)) + np.eye(4))[None] / 20.0
    Ae = Ke + kappa * Me
    rows = np.repeat(mesh.tets, 4, axis=1).ravel()
    cols = np.tile(mesh.tets, (1, 4)).ravel()
    A = sp.csr_matrix((Ae.reshape(-1), (rows, cols)), shape=(mesh.n_nodes, mesh.n_nodes))
    if eliminated is not None:
        el = np.asarray(eliminated, dtype=bool)
        A = A.tocoo()
        keep = (A.row == A.col) | ~(el[A.row] | el[A.col])
        A = sp.csr_matrix((A.data[keep], (A.row[keep], A.col[keep])), shape=A.shape)
    return A

