"""ctypes wrappers over the plain C oracle ``fsi_oracle.c`` (FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every nodal array is float64 ``[n, 4]`` with nodes lexicographic, x fastest.
Physics is passed as a dict with keys rho, mu, dt (None or inf = steady),
C_I (default 36), C_T (default 4), has_s (default False).

Pins (tests/test_oracle_*.py):
  shape, interp      -- exact reproduction of trilinear fields; partition of unity
  locate, cell_hash  -- brute force over all elements on tiny grids
  spread             -- exact adjointness with interp; force conservation
  tau                -- closed-form limits (Stokes, inviscid, convective)
  residual           -- single-element exact integration (4x4x4 Gauss, different
                        points) of the Bazilevs form on fields where 2x2x2 Gauss is
                        exact; Galerkin part on multi-element grids; manufactured
                        solution convergence rates; sum invariants
  jacobian_apply     -- central finite differences of the residual (O(eps^2))
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fsi_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over elements)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
        )
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # FSI_ORACLE_LIB lets the mutation tests load a deliberately broken copy
            L = ctypes.CDLL(os.environ.get("FSI_ORACLE_LIB") or build())
            d = ctypes.POINTER(ctypes.c_double)
            i32 = ctypes.POINTER(ctypes.c_int32)
            i64 = ctypes.POINTER(ctypes.c_int64)
            ci = ctypes.POINTER(ctypes.c_int)
            L.or_shape.argtypes = [d, d, d]
            L.or_tau.argtypes = [d, ctypes.c_double, d, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, d]
            L.or_residual.argtypes = [ci, d, d, d, d, d, ctypes.c_int, d, ctypes.c_int]
            L.or_jacobian_apply.argtypes = [ci, d, d, d, d, d, d, ctypes.c_double,
                                            ctypes.c_double, d, ctypes.c_int]
            L.or_element_jacobian.argtypes = [ci, d, d, d, d, d, ctypes.c_double,
                                              ctypes.c_double, d, i64, ctypes.c_int]
            L.or_locate.argtypes = [ci, d, d, ctypes.c_int64, d, i32, d]
            L.or_locate.restype = ctypes.c_int64
            L.or_residual_x.argtypes = [ci, d, d, d, d, d, ctypes.c_int, d, ctypes.c_int]
            L.or_jacobian_apply_x.argtypes = [ci, d, d, d, d, d, d, ctypes.c_double,
                                              ctypes.c_double, d, ctypes.c_int]
            L.or_element_jacobian_x.argtypes = [ci, d, d, d, d, d, ctypes.c_double,
                                                ctypes.c_double, d, i64, ctypes.c_int]
            L.or_locate_x.argtypes = [ci, d, ctypes.c_int64, d, i32, d]
            L.or_locate_x.restype = ctypes.c_int64
            L.or_cell_hash.argtypes = [ci, ctypes.c_int64, i32, i32, i32]
            L.or_interp.argtypes = [ci, ctypes.c_int64, i32, d, d, d]
            L.or_spread.argtypes = [ci, ctypes.c_int64, i32, d, d, d, d, ctypes.c_int]
            _lib = L
    return _lib


def _p(a, ct=ctypes.c_double):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        assert a.shape == shape, (a.shape, shape)
    return a


class Grid:
    """Structured hex grid of N[k] elements per axis: uniform and axis-aligned
    (spacing h[k] from x0), or mapped when `coords` [n, 3] gives every node's
    position (same node numbering); the operators then take the geometry of
    each Gauss point from the trilinear map."""

    def __init__(self, N, x0=(0.0, 0.0, 0.0), h=None, coords=None):
        if np.isscalar(N):
            N = (int(N),) * 3
        self.N = tuple(int(v) for v in N)
        self.x0 = tuple(float(v) for v in x0)
        if h is None:
            h = tuple(1.0 / v for v in self.N)
        elif np.isscalar(h):
            h = (float(h),) * 3
        self.h = tuple(float(v) for v in h)
        self.coords = None if coords is None else _f64(coords, (self.n_nodes, 3))

    @property
    def n_nodes(self):
        return (self.N[0] + 1) * (self.N[1] + 1) * (self.N[2] + 1)

    @property
    def n_elems(self):
        return self.N[0] * self.N[1] * self.N[2]

    def node_coords(self):
        """[n, 3] coordinates of the nodes in storage order."""
        if self.coords is not None:
            return self.coords.copy()
        ax = [self.x0[k] + self.h[k] * np.arange(self.N[k] + 1) for k in range(3)]
        Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
        return np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)

    def _c(self):
        return (ctypes.c_int * 3)(*self.N), _f64(self.x0), _f64(self.h)


def phys_array(phys):
    """Pack physics for the C oracle: [rho, mu, C_T/dt^2, C_I, has_s]."""
    dt = phys.get("dt")
    C_T = phys.get("C_T", 4.0)
    ct_dt2 = 0.0 if (dt is None or not math.isfinite(dt)) else C_T / (dt * dt)
    return _f64([phys["rho"], phys["mu"], ct_dt2, phys.get("C_I", 36.0),
                 1.0 if phys.get("has_s", False) else 0.0])


def shape(xi):
    """N[8], dN/dxi[8,3] at parent coordinates xi[3]."""
    N = np.zeros(8)
    dN = np.zeros(24)
    lib().or_shape(_p(_f64(xi, (3,))), _p(N), _p(dN))
    return N, dN.reshape(8, 3)


def tau(v, s, h, rho, mu, dt, C_I=36.0, C_T=4.0):
    """(tau_M, tau_C) of Sec. 2.1 for velocity v on a cell of size h."""
    ct_dt2 = 0.0 if (dt is None or not math.isfinite(dt)) else C_T / (dt * dt)
    out = np.zeros(2)
    hh = _f64(h if not np.isscalar(h) else (h, h, h))
    lib().or_tau(_p(_f64(v, (3,))), float(s), _p(hh), float(rho), float(mu), ct_dt2,
                 float(C_I), _p(out))
    return out[0], out[1]


def residual(grid: Grid, phys, U, A, f=None, stab=True, nthreads=0):
    n = grid.n_nodes
    U = _f64(U, (n, 4))
    A = _f64(A, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    R = np.zeros((n, 4))
    Nc, _, h = grid._c()
    if grid.coords is not None:
        lib().or_residual_x(Nc, _p(grid.coords), _p(phys_array(phys)), _p(U), _p(A), _p(f),
                            1 if stab else 0, _p(R), int(nthreads))
        return R
    lib().or_residual(Nc, _p(h), _p(phys_array(phys)), _p(U), _p(A), _p(f),
                      1 if stab else 0, _p(R), int(nthreads))
    return R


def jacobian_apply(grid: Grid, phys, U, A, x, c_a, c_v, f=None, nthreads=0):
    n = grid.n_nodes
    U = _f64(U, (n, 4))
    A = _f64(A, (n, 4))
    x = _f64(x, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    Jx = np.zeros((n, 4))
    Nc, _, h = grid._c()
    if grid.coords is not None:
        lib().or_jacobian_apply_x(Nc, _p(grid.coords), _p(phys_array(phys)), _p(U), _p(A),
                                  _p(f), _p(x), float(c_a), float(c_v), _p(Jx), int(nthreads))
        return Jx
    lib().or_jacobian_apply(Nc, _p(h), _p(phys_array(phys)), _p(U), _p(A), _p(f), _p(x),
                            float(c_a), float(c_v), _p(Jx), int(nthreads))
    return Jx


def element_jacobian(grid: Grid, phys, U, A, c_a, c_v, f=None, nthreads=0):
    """(Ke[E,32,32], conn[E,8]) element tangents of the VMS residual."""
    n, E = grid.n_nodes, grid.n_elems
    U = _f64(U, (n, 4))
    A = _f64(A, (n, 4))
    f = None if f is None else _f64(f, (n, 4))
    Ke = np.zeros((E, 32, 32))
    conn = np.zeros((E, 8), dtype=np.int64)
    Nc, _, h = grid._c()
    if grid.coords is not None:
        lib().or_element_jacobian_x(Nc, _p(grid.coords), _p(phys_array(phys)), _p(U), _p(A),
                                    _p(f), float(c_a), float(c_v), _p(Ke),
                                    _p(conn, ctypes.c_int64), int(nthreads))
        return Ke, conn
    lib().or_element_jacobian(Nc, _p(h), _p(phys_array(phys)), _p(U), _p(A), _p(f),
                              float(c_a), float(c_v), _p(Ke), _p(conn, ctypes.c_int64),
                              int(nthreads))
    return Ke, conn


def locate(grid: Grid, X):
    """(elem[m] int32, xi[m,3], n_outside) for points X[m,3]."""
    X = _f64(X)
    m = X.shape[0]
    elem = np.zeros(m, dtype=np.int32)
    xi = np.zeros((m, 3))
    Nc, x0, h = grid._c()
    if grid.coords is not None:
        nout = lib().or_locate_x(Nc, _p(grid.coords), m, _p(X), _p(elem, ctypes.c_int32), _p(xi))
        return elem, xi, int(nout)
    nout = lib().or_locate(Nc, _p(x0), _p(h), m, _p(X), _p(elem, ctypes.c_int32), _p(xi))
    return elem, xi, int(nout)


def cell_hash(grid: Grid, elem):
    """(cell_start[E+1] int32, perm[m] int32): stable counting sort by cell."""
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    m = elem.shape[0]
    cs = np.zeros(grid.n_elems + 1, dtype=np.int32)
    perm = np.zeros(m, dtype=np.int32)
    Nc, _, _ = grid._c()
    lib().or_cell_hash(Nc, m, _p(elem, ctypes.c_int32), _p(cs, ctypes.c_int32),
                       _p(perm, ctypes.c_int32))
    return cs, perm


def interp(grid: Grid, elem, xi, U):
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    m = elem.shape[0]
    xi = _f64(xi, (m, 3))
    U = _f64(U, (grid.n_nodes, 4))
    u = np.zeros((m, 3))
    Nc, _, _ = grid._c()
    lib().or_interp(Nc, m, _p(elem, ctypes.c_int32), _p(xi), _p(U), _p(u))
    return u


def spread(grid: Grid, elem, xi, lam, w=None, F=None, accumulate=False):
    elem = np.ascontiguousarray(elem, dtype=np.int32)
    m = elem.shape[0]
    xi = _f64(xi, (m, 3))
    lam = _f64(lam, (m, 3))
    w = None if w is None else _f64(w, (m,))
    if F is None:
        F = np.zeros((grid.n_nodes, 4))
    else:
        F = _f64(F, (grid.n_nodes, 4)).copy()
    Nc, _, _ = grid._c()
    lib().or_spread(Nc, m, _p(elem, ctypes.c_int32), _p(xi), _p(lam), _p(w), _p(F),
                    1 if accumulate else 0)
    return F
