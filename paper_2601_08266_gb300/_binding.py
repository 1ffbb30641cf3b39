"""Thin ctypes binding of libfsi (include/fsi.h).

Argument marshalling only: every operator runs in the CUDA library.  Array
arguments are torch tensors on the mesh's device (contiguous; float64 or
float32 as the precision says; int32 for indices); ``None`` maps to NULL.
There is no CPU fallback: if the library cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

FSI_OK, FSI_ERR_ARG, FSI_ERR_CUDA, FSI_ERR_OOM, FSI_ERR_OUTSIDE = 0, 1, 2, 3, 4
FSI_ERR_NOCONV, FSI_ERR_TIMEOUT, FSI_ERR_NAN = 5, 6, 7
FSI_F64, FSI_F32, FSI_DF64 = 0, 1, 2
STATUS_NAMES = {0: "FSI_OK", 1: "FSI_ERR_ARG", 2: "FSI_ERR_CUDA", 3: "FSI_ERR_OOM",
                4: "FSI_ERR_OUTSIDE", 5: "FSI_ERR_NOCONV", 6: "FSI_ERR_TIMEOUT",
                7: "FSI_ERR_NAN"}


class FsiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fsi_grid(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int32 * 3), ("x0", ctypes.c_double * 3),
                ("h", ctypes.c_double * 3)]


class fsi_physics(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("mu", ctypes.c_double), ("dt", ctypes.c_double),
                ("rho_inf", ctypes.c_double), ("C_I", ctypes.c_double),
                ("C_T", ctypes.c_double), ("has_s", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fsi_step_state(ctypes.Structure):
    _fields_ = [("y", ctypes.c_void_p), ("Vn", ctypes.c_void_p), ("An", ctypes.c_void_p),
                ("s", ctypes.c_void_p), ("f", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("yD", ctypes.c_void_p), ("m", ctypes.c_int64), ("elem", ctypes.c_void_p),
                ("cell_start", ctypes.c_void_p), ("perm", ctypes.c_void_p),
                ("xi", ctypes.c_void_p), ("w", ctypes.c_void_p), ("drho_s", ctypes.c_double),
                ("k_s", ctypes.c_double), ("g_s", ctypes.c_double * 3),
                ("body", ctypes.c_void_p), ("us", ctypes.c_void_p), ("vs", ctypes.c_void_p),
                ("as_", ctypes.c_void_p)]


class fsi_newton_opts(ctypes.Structure):
    _fields_ = [("mixed", ctypes.c_int32), ("restart", ctypes.c_int32),
                ("max_newton", ctypes.c_int32), ("max_krylov", ctypes.c_int32),
                ("newton_rtol", ctypes.c_double), ("krylov_rtol", ctypes.c_double),
                ("r_ref", ctypes.c_double), ("precond_every", ctypes.c_int32),
                ("precond", ctypes.c_int32), ("residual_prec", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("R0", ctypes.c_void_p)]


class fsi_newton_report(ctypes.Structure):
    _fields_ = [("newton_iters", ctypes.c_int32), ("krylov_iters", ctypes.c_int32),
                ("r0", ctypes.c_double), ("r_final", ctypes.c_double),
                ("r_ref", ctypes.c_double), ("seconds", ctypes.c_double),
                ("converged", ctypes.c_int32), ("precond_builds", ctypes.c_int32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fsi_guess_report(ctypes.Structure):
    _fields_ = [("r_fallback", ctypes.c_double), ("r_learned", ctypes.c_double),
                ("r_combined", ctypes.c_double), ("c_d1", ctypes.c_double),
                ("c_d2", ctypes.c_double), ("c_net", ctypes.c_double),
                ("used", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("r_history_fit", ctypes.c_double)]


class fsi_batch_item(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("A", ctypes.c_void_p), ("f", ctypes.c_void_p),
                ("x", ctypes.c_void_p), ("R", ctypes.c_void_p), ("Jx", ctypes.c_void_p),
                ("m", ctypes.c_int64), ("elem", ctypes.c_void_p),
                ("cell_start", ctypes.c_void_p), ("perm", ctypes.c_void_p),
                ("xi", ctypes.c_void_p), ("lam", ctypes.c_void_p), ("w", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("F", ctypes.c_void_p), ("X", ctypes.c_void_p)]


_NT = 64


class fsi_tune_report(ctypes.Structure):
    _fields_ = [("bx", ctypes.c_int32), ("by", ctypes.c_int32), ("bz", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("n_candidates", ctypes.c_int32), ("seconds", ctypes.c_double),
                ("cand_bx", ctypes.c_int32 * _NT), ("cand_by", ctypes.c_int32 * _NT),
                ("cand_bz", ctypes.c_int32 * _NT), ("cand_ctas", ctypes.c_int32 * _NT),
                ("cand_seconds", ctypes.c_double * _NT)]


FSI_BATCH_PER_INSTANCE, FSI_BATCH_PERSISTENT, FSI_BATCH_GRAPH = 0, 1, 2

_lock = threading.Lock()
_lib = None

_VP = ctypes.c_void_p
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_SIGS = {
    "fsi_mesh_create": ([ctypes.POINTER(fsi_grid), ctypes.POINTER(fsi_physics), _INT, _VP,
                         ctypes.POINTER(_VP)], _INT),
    "fsi_mesh_destroy": ([_VP], None),
    "fsi_mesh_set_stream": ([_VP, _VP], _INT),
    "fsi_mesh_set_physics": ([_VP, ctypes.POINTER(fsi_physics)], _INT),
    "fsi_mesh_sizes": ([_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)], _INT),
    "fsi_last_error": ([], ctypes.c_char_p),
    "fsi_stage": ([_VP, _INT, _VP, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_residual": ([_VP, _INT, _VP, _VP, _VP, _VP], _INT),
    "fsi_jacobian_apply": ([_VP, _INT, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_locate": ([_VP, _I64, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_I64), _INT], _INT),
    "fsi_dlm_interp": ([_VP, _INT, _I64, _VP, _VP, _VP, _VP], _INT),
    "fsi_dlm_spread": ([_VP, _INT, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _INT], _INT),
    "fsi_measure_fma_peak": ([_INT, _INT, ctypes.POINTER(ctypes.c_double)], _INT),
    "fsi_multi_dot": ([_INT, _INT, _I64, _INT, _VP, _I64, _VP, _VP], _INT),
    "fsi_measure_blas1": ([_INT, _INT, _I64, _INT, _INT, ctypes.POINTER(ctypes.c_double),
                           ctypes.POINTER(ctypes.c_double)], _INT),
    "fsi_coupled_residual": ([_VP, _INT, ctypes.POINTER(fsi_step_state), _VP], _INT),
    "fsi_coupled_jacobian_apply": ([_VP, _INT, ctypes.POINTER(fsi_step_state), _VP, _VP], _INT),
    "fsi_block_diagonal": ([_VP, _INT, ctypes.POINTER(fsi_step_state), _VP], _INT),
    "fsi_newton_step": ([_VP, ctypes.POINTER(fsi_newton_opts), ctypes.POINTER(fsi_step_state),
                         ctypes.POINTER(fsi_newton_report)], _INT),
    "fsi_solid_create": ([_VP, _I64, _I64, _VP, _VP, ctypes.c_double, ctypes.c_double,
                          ctypes.c_double, ctypes.POINTER(_VP)], _INT),
    "fsi_solid_destroy": ([_VP], None),
    "fsi_solid_residual": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_solid_tangent_apply": ([_VP, _INT, _VP, _VP, _VP, _VP], _INT),
    "fsi_solid_stage": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_solid_advance": ([_VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_solid_positions": ([_VP, _VP, _VP], _INT),
    "fsi_mesh_set_coordinates": ([_VP, _VP], _INT),
    "fsi_wait_selftest": ([_INT, ctypes.POINTER(_INT), ctypes.POINTER(ctypes.c_double)], _INT),
    "fsi_mesh_create_tet": ([_I64, _VP, _I64, _VP, ctypes.POINTER(fsi_physics), _INT, _VP,
                             ctypes.POINTER(_VP)], _INT),
    "fsi_tetmesh_create": ([_I64, _VP, _I64, _VP, ctypes.POINTER(fsi_physics), _INT, _VP,
                            ctypes.POINTER(_VP)], _INT),
    "fsi_tetmesh_destroy": ([_VP], None),
    "fsi_tet_residual": ([_VP, _INT, _VP, _VP, _VP, _VP], _INT),
    "fsi_tet_jacobian_apply": ([_VP, _INT, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_tet_locate": ([_VP, _I64, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(_I64)], _INT),
    "fsi_tet_interp": ([_VP, _INT, _I64, _VP, _VP, _VP, _VP], _INT),
    "fsi_tet_spread": ([_VP, _INT, _I64, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _INT], _INT),
    "fsi_interface_scaling": ([_VP, _VP, ctypes.c_double, _INT, _VP], _INT),
    "fsi_pressure_levels": ([_VP, ctypes.POINTER(ctypes.c_int32), _VP], _INT),
    "fsi_pressure_set_faces": ([_VP, ctypes.POINTER(ctypes.c_int32)], _INT),
    "fsi_pressure_level_sizes": ([_VP, ctypes.POINTER(ctypes.c_int32),
                                  ctypes.POINTER(ctypes.c_int64)], _INT),
    "fsi_pressure_set_eliminated": ([_VP, _VP], _INT),
    "fsi_pressure_use_amg": ([_VP, ctypes.c_int32], _INT),
    "fsi_pressure_apply": ([_VP, _INT, _INT, _VP, _VP], _INT),
    "fsi_pressure_restrict": ([_VP, _INT, _INT, _VP, _VP], _INT),
    "fsi_pressure_prolong_add": ([_VP, _INT, _INT, _VP, _VP], _INT),
    "fsi_pressure_smooth": ([_VP, _INT, _INT, _INT, _VP, _VP, _INT], _INT),
    "fsi_pressure_vcycle": ([_VP, _INT, _VP, _VP], _INT),
    "fsi_locate_noalloc": ([ctypes.POINTER(fsi_grid), _I64, _VP, _VP, _VP, _VP, _VP,
                            ctypes.POINTER(_I64), _INT, _INT, _VP], _INT),
    "fsi_mlp_create": ([_INT, _VP, _I64, ctypes.POINTER(_VP)], _INT),
    "fsi_mlp_destroy": ([_VP], None),
    "fsi_mlp_check": ([_VP], _INT),
    "fsi_mlp_num_params": ([], _I64),
    "fsi_mlp_forward": ([_VP, _VP, _VP, _I64, _VP], _INT),
    "fsi_mlp_loss_grad": ([_VP, _VP, _VP, _VP, _I64, _VP, _VP], _INT),
    "fsi_mlp_adam": ([_VP, _VP, _VP, _VP, _VP, _INT, ctypes.c_float, ctypes.c_float,
                      ctypes.c_float, ctypes.c_float], _INT),
    "fsi_mlp_features": ([_VP, _VP, _VP, _VP, _VP, _VP, _I64, _VP, _VP, _VP], _INT),
    "fsi_mlp_predict": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP], _INT),
    "fsi_mlp_guess": ([_VP, _VP, _VP, _VP, _VP, _VP, _VP, ctypes.POINTER(fsi_step_state), _VP,
                       _VP, _VP, _INT, _INT, _VP, ctypes.POINTER(fsi_guess_report)], _INT),
    "fsi_advance_history": ([_VP, _INT, _VP, _VP, _VP], _INT),
    "fsi_batch_create": ([ctypes.POINTER(_VP), ctypes.POINTER(fsi_batch_item), _INT, _INT, _VP,
                          ctypes.POINTER(_VP)], _INT),
    "fsi_batch_destroy": ([_VP], None),
    "fsi_batch_run": ([_VP, _INT], _INT),
    "fsi_batch_time": ([_VP, _INT, _INT, ctypes.POINTER(ctypes.c_double)], _INT),
    "fsi_batch_autotune": ([_VP, _INT, ctypes.POINTER(fsi_tune_report)], _INT),
    "fsi_mesh_set_brick": ([_VP, _INT, _INT, _INT, _INT, _INT, _INT], _INT),
    "fsi_mesh_autotune": ([_VP, _INT, _INT, _INT, ctypes.POINTER(fsi_tune_report)], _INT),
    "fsi_residual_jacobian_apply": ([_VP, _INT, _VP, _VP, _VP, _VP, _VP, _VP], _INT),
}


def library_path() -> str:
    return _build.LIB


def lib():
    """Load (building first if needed) libfsi.so and declare its signatures."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            L = ctypes.CDLL(path)
            for name, (args, res) in _SIGS.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(st):
    if st != FSI_OK:
        raise FsiError(st, lib().fsi_last_error().decode())


def _ptr(t, dtype=None):
    if t is None:
        return None
    import torch
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch tensor")
    if not t.is_cuda:
        raise ValueError("array arguments must be CUDA tensors (device memory)")
    if not t.is_contiguous():
        raise ValueError("array arguments must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _prec_dtype(prec):
    import torch
    return torch.float32 if prec == FSI_F32 else torch.float64


class Mesh:
    """Owner of an fsi_mesh handle."""

    def __init__(self, N, x0=(0.0, 0.0, 0.0), h=None, rho=1.0, mu=0.01, dt=1e-3,
                 rho_inf=0.5, C_I=36.0, C_T=4.0, has_s=False, device=0, stream=None):
        import torch
        if isinstance(N, int):
            N = (N, N, N)
        if h is None:
            h = tuple(1.0 / v for v in N)
        elif isinstance(h, (int, float)):
            h = (float(h),) * 3
        self.N, self.x0, self.h = tuple(N), tuple(x0), tuple(h)
        self.device = device
        g = fsi_grid((ctypes.c_int32 * 3)(*N), (ctypes.c_double * 3)(*x0),
                     (ctypes.c_double * 3)(*h))
        self.phys = fsi_physics(rho, mu, dt, rho_inf, C_I, C_T, 1 if has_s else 0, 0)
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._stream = stream
        out = ctypes.c_void_p()
        _check(lib().fsi_mesh_create(ctypes.byref(g), ctypes.byref(self.phys), device,
                                     ctypes.c_void_p(stream), ctypes.byref(out)))
        self.handle = out

    @property
    def n_nodes(self):
        return (self.N[0] + 1) * (self.N[1] + 1) * (self.N[2] + 1)

    @property
    def n_elems(self):
        return self.N[0] * self.N[1] * self.N[2]

    def set_stream(self, stream):
        self._stream = stream
        _check(lib().fsi_mesh_set_stream(self.handle, ctypes.c_void_p(stream)))

    def set_coordinates(self, X):
        """Node coordinates [n, 3] FP64 (device) of a mapped grid, None = uniform."""
        fsi_mesh_set_coordinates(self, X)

    def set_physics(self, **kw):
        for k, v in kw.items():
            setattr(self.phys, k, v)
        _check(lib().fsi_mesh_set_physics(self.handle, ctypes.byref(self.phys)))

    def close(self):
        if getattr(self, "handle", None):
            lib().fsi_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------- C-ABI mirrors
def fsi_stage(mesh: Mesh, prec, y, Vn, An, s, U, A):
    dt = _prec_dtype(prec)
    _check(lib().fsi_stage(mesh.handle, prec, _ptr(y, dt), _ptr(Vn, dt), _ptr(An, dt),
                           _ptr(s, dt), _ptr(U, dt), _ptr(A, dt)))


def fsi_residual(mesh: Mesh, prec, U, A, f, R):
    dt = _prec_dtype(prec)
    _check(lib().fsi_residual(mesh.handle, prec, _ptr(U, dt), _ptr(A, dt), _ptr(f, dt),
                              _ptr(R, dt)))


def fsi_residual_jacobian_apply(mesh: Mesh, prec, U, A, f, x, R, Jx):
    dt = _prec_dtype(prec)
    _check(lib().fsi_residual_jacobian_apply(mesh.handle, prec, _ptr(U, dt), _ptr(A, dt),
                                             _ptr(f, dt), _ptr(x, dt), _ptr(R, dt),
                                             _ptr(Jx, dt)))


def fsi_jacobian_apply(mesh: Mesh, prec, U, A, f, x, Jx):
    dt = _prec_dtype(prec)
    _check(lib().fsi_jacobian_apply(mesh.handle, prec, _ptr(U, dt), _ptr(A, dt), _ptr(f, dt),
                                    _ptr(x, dt), _ptr(Jx, dt)))


def fsi_locate(mesh: Mesh, X, elem, xi, cell_start=None, perm=None, want_outside=True,
               strict=False):
    import torch
    m = 0 if X is None else X.shape[0]
    nout = _I64(0)
    _check(lib().fsi_locate(mesh.handle, m, _ptr(X, torch.float64), _ptr(elem, torch.int32),
                            _ptr(xi, torch.float64), _ptr(cell_start, torch.int32),
                            _ptr(perm, torch.int32),
                            ctypes.byref(nout) if want_outside else None,
                            1 if strict else 0))
    return int(nout.value) if want_outside else None


def fsi_dlm_interp(mesh: Mesh, prec, elem, xi, U, u):
    import torch
    dt = _prec_dtype(prec)
    _check(lib().fsi_dlm_interp(mesh.handle, prec, elem.shape[0], _ptr(elem, torch.int32),
                                _ptr(xi, dt), _ptr(U, dt), _ptr(u, dt)))


def fsi_dlm_spread(mesh: Mesh, prec, elem, xi, cell_start, perm, lam, w, F, accumulate):
    import torch
    dt = _prec_dtype(prec)
    m = elem.shape[0] if elem is not None else lam.shape[0]
    _check(lib().fsi_dlm_spread(mesh.handle, prec, m, _ptr(elem, torch.int32), _ptr(xi, dt),
                                _ptr(cell_start, torch.int32), _ptr(perm, torch.int32),
                                _ptr(lam, dt), _ptr(w, dt), _ptr(F, dt),
                                1 if accumulate else 0))


class TetMesh:
    """Owner of an fsi_tetmesh handle: X [n, 3] float64 and tets [E, 4] int32
    device tensors (copied by the library)."""

    def __init__(self, X, tets, rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, C_I=36.0, C_T=4.0,
                 has_s=False, device=0, stream=None):
        import torch
        self.n_nodes, self.n_elems = int(X.shape[0]), int(tets.shape[0])
        if tuple(X.shape) != (self.n_nodes, 3) or tuple(tets.shape) != (self.n_elems, 4):
            raise ValueError("X must be [n, 3] and tets [E, 4]")
        self.device = device
        self.phys = fsi_physics(rho, mu, dt, rho_inf, C_I, C_T, 1 if has_s else 0, 0)
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        out = ctypes.c_void_p()
        _check(lib().fsi_tetmesh_create(self.n_nodes, _ptr(X, torch.float64), self.n_elems,
                                        _ptr(tets, torch.int32), ctypes.byref(self.phys), device,
                                        ctypes.c_void_p(stream), ctypes.byref(out)))
        self.handle = out

    def close(self):
        if getattr(self, "handle", None):
            lib().fsi_tetmesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MeshTet(Mesh):
    """An fsi_mesh handle backed by a tetrahedral mesh (fsi_mesh_create_tet):
    the step's entry points (fsi_residual, fsi_locate, fsi_newton_step, ...)
    accept it like a structured-grid Mesh.  X [n, 3] float64 and tets [E, 4]
    int32 device tensors."""

    def __init__(self, X, tets, rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, C_I=36.0, C_T=4.0,
                 has_s=False, device=0, stream=None):
        import torch
        self._n, self._E = int(X.shape[0]), int(tets.shape[0])
        if tuple(X.shape) != (self._n, 3) or tuple(tets.shape) != (self._E, 4):
            raise ValueError("X must be [n, 3] and tets [E, 4]")
        self.N = None
        self.device = device
        self.phys = fsi_physics(rho, mu, dt, rho_inf, C_I, C_T, 1 if has_s else 0, 0)
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        self._stream = stream
        out = ctypes.c_void_p()
        _check(lib().fsi_mesh_create_tet(self._n, _ptr(X, torch.float64), self._E,
                                         _ptr(tets, torch.int32), ctypes.byref(self.phys), device,
                                         ctypes.c_void_p(stream), ctypes.byref(out)))
        self.handle = out

    @property
    def n_nodes(self):
        return self._n

    @property
    def n_elems(self):
        return self._E


def fsi_tet_residual(mesh: TetMesh, prec, U, A, f, R):
    dt = _prec_dtype(prec)
    _check(lib().fsi_tet_residual(mesh.handle, prec, _ptr(U, dt), _ptr(A, dt), _ptr(f, dt),
                                  _ptr(R, dt)))


def fsi_tet_jacobian_apply(mesh: TetMesh, prec, U, A, f, x, Jx):
    dt = _prec_dtype(prec)
    _check(lib().fsi_tet_jacobian_apply(mesh.handle, prec, _ptr(U, dt), _ptr(A, dt),
                                        _ptr(f, dt), _ptr(x, dt), _ptr(Jx, dt)))


def fsi_tet_locate(mesh: TetMesh, P, elem, lam, cell_start=None, perm=None, want_outside=True):
    import torch
    m = 0 if P is None else P.shape[0]
    nout = _I64(0)
    _check(lib().fsi_tet_locate(mesh.handle, m, _ptr(P, torch.float64), _ptr(elem, torch.int32),
                                _ptr(lam, torch.float64), _ptr(cell_start, torch.int32),
                                _ptr(perm, torch.int32),
                                ctypes.byref(nout) if want_outside else None))
    return int(nout.value) if want_outside else None


def fsi_tet_interp(mesh: TetMesh, prec, elem, lam, U, u):
    import torch
    dt = _prec_dtype(prec)
    _check(lib().fsi_tet_interp(mesh.handle, prec, elem.shape[0], _ptr(elem, torch.int32),
                                _ptr(lam, dt), _ptr(U, dt), _ptr(u, dt)))


def fsi_tet_spread(mesh: TetMesh, prec, elem, lam, cell_start, perm, lamv, w, F, accumulate):
    import torch
    dt = _prec_dtype(prec)
    m = elem.shape[0] if elem is not None else lamv.shape[0]
    _check(lib().fsi_tet_spread(mesh.handle, prec, m, _ptr(elem, torch.int32), _ptr(lam, dt),
                                _ptr(cell_start, torch.int32), _ptr(perm, torch.int32),
                                _ptr(lamv, dt), _ptr(w, dt), _ptr(F, dt),
                                1 if accumulate else 0))


def fsi_wait_selftest(device=0):
    """(timed_out, seconds) of the planted never-ending wait (see fsi.h)."""
    t = _INT(0)
    sec = ctypes.c_double(0.0)
    _check(lib().fsi_wait_selftest(device, ctypes.byref(t), ctypes.byref(sec)))
    return bool(t.value), sec.value


def fsi_measure_fma_peak(device, prec):
    out = ctypes.c_double(0.0)
    _check(lib().fsi_measure_fma_peak(device, prec, ctypes.byref(out)))
    return out.value


def fsi_multi_dot(prec, V, w, out, device=0):
    """out[k] = V[k] . w (the Krylov multi-dot; V [nvec, len], w [len], out
    float64 [nvec], all device tensors)."""
    import torch
    dt = _prec_dtype(prec)
    nvec, length = V.shape
    _check(lib().fsi_multi_dot(device, prec, int(length), int(nvec), _ptr(V, dt), int(length),
                               _ptr(w, dt), _ptr(out, torch.float64)))


def fsi_measure_blas1(device, prec, length, nvec, reps=10):
    """(seconds per multi-dot, seconds per multi-update) of the Krylov
    BLAS-1 kernels on nvec basis vectors of `length` entries."""
    d, a = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(lib().fsi_measure_blas1(device, prec, int(length), int(nvec), int(reps),
                                   ctypes.byref(d), ctypes.byref(a)))
    return d.value, a.value


class StepState:
    """Owns the torch tensors behind an fsi_step_state (all FP64 on the device)."""

    def __init__(self, y, Vn, An, s=None, f=None, mask=None, yD=None, elem=None, xi=None,
                 cell_start=None, perm=None, w=None, drho_s=0.5, k_s=0.0, g_s=(0.0, 0.0, 0.0),
                 body=None, us=None, vs=None, as_=None):
        import torch
        self.t = dict(y=y, Vn=Vn, An=An, s=s, f=f, mask=mask, yD=yD, elem=elem, xi=xi,
                      cell_start=cell_start, perm=perm, w=w, us=us, vs=vs, as_=as_)
        self.body = body
        m = 0 if elem is None else int(elem.shape[0])
        f64 = torch.float64
        self.c = fsi_step_state(
            _ptr(y, f64), _ptr(Vn, f64), _ptr(An, f64), _ptr(s, f64), _ptr(f, f64),
            _ptr(mask, torch.uint8), _ptr(yD, f64), m, _ptr(elem, torch.int32),
            _ptr(cell_start, torch.int32), _ptr(perm, torch.int32), _ptr(xi, f64),
            _ptr(w, f64), float(drho_s), float(k_s), (ctypes.c_double * 3)(*g_s),
            None if body is None else body.handle.value, _ptr(us, f64), _ptr(vs, f64),
            _ptr(as_, f64))


def fsi_coupled_residual(mesh: Mesh, st: StepState, R, prec=FSI_F64):
    import torch
    _check(lib().fsi_coupled_residual(mesh.handle, int(prec), ctypes.byref(st.c),
                                      _ptr(R, torch.float64)))


def fsi_coupled_jacobian_apply(mesh: Mesh, prec, st: StepState, x, Jx):
    dt = _prec_dtype(prec)
    _check(lib().fsi_coupled_jacobian_apply(mesh.handle, prec, ctypes.byref(st.c), _ptr(x, dt),
                                            _ptr(Jx, dt)))


def fsi_block_diagonal(mesh: Mesh, prec, st: StepState, blocks):
    dt = _prec_dtype(prec)
    _check(lib().fsi_block_diagonal(mesh.handle, prec, ctypes.byref(st.c), _ptr(blocks, dt)))


PRECOND_BLOCK_JACOBI, PRECOND_SCHUR = 0, 1


def fsi_newton_step(mesh: Mesh, st: StepState, mixed=True, restart=50, max_newton=10,
                    max_krylov=1000, newton_rtol=1e-8, krylov_rtol=1e-3, r_ref=0.0,
                    precond_every=0, precond=PRECOND_SCHUR, residual_prec=FSI_F64, check=True,
                    R0=None):
    """Returns (status, report dict); raises on error when check is True.
    R0: optional FP64 [n, 4] device tensor holding R(st.y) in residual_prec."""
    import torch
    if R0 is not None and R0.numel() != 4 * mesh.n_nodes:
        raise ValueError("R0 must hold [n_nodes, 4] values")
    o = fsi_newton_opts(1 if mixed else 0, restart, max_newton, max_krylov, newton_rtol,
                        krylov_rtol, r_ref, precond_every, int(precond), int(residual_prec), 0,
                        _ptr(R0, torch.float64) if R0 is not None else None)
    rep = fsi_newton_report()
    st_code = lib().fsi_newton_step(mesh.handle, ctypes.byref(o), ctypes.byref(st.c),
                                    ctypes.byref(rep))
    if check:
        _check(st_code)
    return st_code, rep.as_dict()


def fsi_locate_noalloc(N, x0, h, X, elem, xi, cell_start=None, perm=None, want_outside=True,
                       strict=False, device=0, stream=None):
    """Point location that allocates no device memory (see include/fsi.h)."""
    import torch
    if isinstance(N, int):
        N = (N, N, N)
    g = fsi_grid((ctypes.c_int32 * 3)(*N), (ctypes.c_double * 3)(*x0), (ctypes.c_double * 3)(*h))
    if stream is None:
        stream = torch.cuda.current_stream(device).cuda_stream
    m = 0 if X is None else X.shape[0]
    nout = _I64(0)
    _check(lib().fsi_locate_noalloc(ctypes.byref(g), m, _ptr(X, torch.float64),
                                    _ptr(elem, torch.int32), _ptr(xi, torch.float64),
                                    _ptr(cell_start, torch.int32), _ptr(perm, torch.int32),
                                    ctypes.byref(nout) if want_outside else None,
                                    1 if strict else 0, device, ctypes.c_void_p(stream)))
    return int(nout.value) if want_outside else None


class Mlp:
    """Owner of an fsi_mlp handle (activation scratch for max_batch rows)."""

    def __init__(self, max_batch, device=0, stream=None):
        import torch
        if stream is None:
            stream = torch.cuda.current_stream(device).cuda_stream
        out = ctypes.c_void_p()
        _check(lib().fsi_mlp_create(device, ctypes.c_void_p(stream), int(max_batch),
                                    ctypes.byref(out)))
        self.handle = out
        self.max_batch = int(max_batch)

    def check(self):
        """Raise FsiError(FSI_ERR_TIMEOUT) if a tensor-core wait of an earlier
        call ran out (synchronises the device)."""
        _check(lib().fsi_mlp_check(self.handle))

    def close(self):
        if getattr(self, "handle", None):
            lib().fsi_mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fsi_mlp_num_params():
    return int(lib().fsi_mlp_num_params())


def fsi_mlp_forward(mlp: Mlp, params, X, out):
    import torch
    f = torch.float32
    _check(lib().fsi_mlp_forward(mlp.handle, _ptr(params, f), _ptr(X, f), X.shape[0],
                                 _ptr(out, f)))


def fsi_mlp_loss_grad(mlp: Mlp, params, X, T, loss, grad):
    import torch
    f = torch.float32
    _check(lib().fsi_mlp_loss_grad(mlp.handle, _ptr(params, f), _ptr(X, f), _ptr(T, f),
                                   X.shape[0], _ptr(loss, f), _ptr(grad, f)))


def fsi_mlp_adam(mlp: Mlp, params, grad, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    import torch
    f = torch.float32
    _check(lib().fsi_mlp_adam(mlp.handle, _ptr(params, f), _ptr(grad, f), _ptr(m, f), _ptr(v, f),
                              int(step), lr, beta1, beta2, eps))


def fsi_mlp_features(mesh: Mesh, Vn, y, d1, d2, idx, in_mean, in_std, X):
    import torch
    d, f = torch.float64, torch.float32
    k = 0 if idx is None else idx.shape[0]
    _check(lib().fsi_mlp_features(mesh.handle, _ptr(Vn, d), _ptr(y, d), _ptr(d1, d), _ptr(d2, d),
                                  _ptr(idx, torch.int32), k, _ptr(in_mean, f), _ptr(in_std, f),
                                  _ptr(X, f)))


def fsi_mlp_predict(mlp: Mlp, mesh: Mesh, params, in_mean, in_std, out_mean, out_std, Vn, y, d1,
                    d2, y0):
    import torch
    d, f = torch.float64, torch.float32
    _check(lib().fsi_mlp_predict(mlp.handle, mesh.handle, _ptr(params, f), _ptr(in_mean, f),
                                 _ptr(in_std, f), _ptr(out_mean, f), _ptr(out_std, f),
                                 _ptr(Vn, d), _ptr(y, d), _ptr(d1, d), _ptr(d2, d), _ptr(y0, d)))


def fsi_advance_history(mesh: Mesh, prec, y, Vn, An):
    dt = _prec_dtype(prec)
    _check(lib().fsi_advance_history(mesh.handle, prec, _ptr(y, dt), _ptr(Vn, dt), _ptr(An, dt)))


def fsi_mlp_guess(mlp: Mlp, mesh: Mesh, params, in_mean, in_std, out_mean, out_std,
                  st: "StepState", yn, d1, d2, fallback, work, judge_prec=FSI_F64):
    import torch
    d, f = torch.float64, torch.float32
    if work.numel() < 5 * 4 * mesh.n_nodes:
        raise ValueError("fsi_mlp_guess: work must hold [5, n_nodes, 4] float64 values")
    rep = fsi_guess_report()
    _check(lib().fsi_mlp_guess(mlp.handle, mesh.handle, _ptr(params, f), _ptr(in_mean, f),
                               _ptr(in_std, f), _ptr(out_mean, f), _ptr(out_std, f),
                               ctypes.byref(st.c), _ptr(yn, d), _ptr(d1, d), _ptr(d2, d),
                               int(fallback), int(judge_prec), _ptr(work, d),
                               ctypes.byref(rep)))
    return {k: getattr(rep, k) for k, _ in fsi_guess_report._fields_ if k != "reserved"}


def _prec_of(t):
    import torch
    if t.dtype == torch.float64:
        return FSI_F64
    if t.dtype == torch.float32:
        return FSI_F32
    raise TypeError("pressure vectors must be float64 or float32")


def fsi_pressure_levels(mesh: Mesh):
    """List of (Nx, Ny, Nz) per level of the pressure hierarchy."""
    n = ctypes.c_int32(0)
    buf = (ctypes.c_int32 * 48)()
    _check(lib().fsi_pressure_levels(mesh.handle, ctypes.byref(n), buf))
    return [tuple(buf[3 * l + d] for d in range(3)) for l in range(n.value)]


class Solid:
    """Owner of an fsi_solid handle (hyperelastic immersed solid, Q1 hexahedra)."""

    def __init__(self, mesh: Mesh, X, conn, rho_s, mu_s, lambda_s):
        import torch
        self.mesh = mesh
        self.X = X
        self.ns, self.es = int(X.shape[0]), int(conn.shape[0])
        h = _VP()
        _check(lib().fsi_solid_create(mesh.handle, self.ns, self.es, _ptr(X, torch.float64),
                                      _ptr(conn, torch.int32), float(rho_s), float(mu_s),
                                      float(lambda_s), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            lib().fsi_solid_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fsi_solid_residual(body: Solid, u_af, v_af, a_am, u_n, g, R):
    import torch
    d = torch.float64
    g_arr = None if g is None else (ctypes.c_double * 3)(*g)   # alive during the call
    g_ptr = None if g_arr is None else ctypes.cast(g_arr, ctypes.c_void_p)
    _check(lib().fsi_solid_residual(body.handle, _ptr(u_af, d), _ptr(v_af, d), _ptr(a_am, d),
                                    _ptr(u_n, d), g_ptr, _ptr(R, d)))


def fsi_solid_tangent_apply(body: Solid, prec, u_af, u_n, x, Jx):
    import torch
    dt = _prec_dtype(prec)
    _check(lib().fsi_solid_tangent_apply(body.handle, prec, _ptr(u_af, dt),
                                         _ptr(u_n, torch.float64), _ptr(x, dt), _ptr(Jx, dt)))


def fsi_solid_stage(body: Solid, u, v, a, a_next, u_af, v_af, a_am):
    import torch
    d = torch.float64
    _check(lib().fsi_solid_stage(body.handle, _ptr(u, d), _ptr(v, d), _ptr(a, d),
                                 _ptr(a_next, d), _ptr(u_af, d), _ptr(v_af, d), _ptr(a_am, d)))


def fsi_solid_advance(body: Solid, u, v, a, a_next):
    import torch
    d = torch.float64
    _check(lib().fsi_solid_advance(body.handle, _ptr(u, d), _ptr(v, d), _ptr(a, d),
                                   _ptr(a_next, d)))


def fsi_solid_positions(body: Solid, u, x):
    import torch
    d = torch.float64
    _check(lib().fsi_solid_positions(body.handle, _ptr(u, d), _ptr(x, d)))


def fsi_mesh_set_coordinates(mesh: Mesh, X):
    import torch
    if X is not None and X.numel() != 3 * mesh.n_nodes:
        raise ValueError("coordinates must be [n_nodes, 3]")
    _check(lib().fsi_mesh_set_coordinates(mesh.handle, _ptr(X, torch.float64)))


def fsi_interface_scaling(mesh: Mesh, cell_start, s_band, layers, s):
    import torch
    _check(lib().fsi_interface_scaling(mesh.handle, _ptr(cell_start, torch.int32), float(s_band),
                                       int(layers), _ptr(s, torch.float64)))


def fsi_pressure_set_faces(mesh: Mesh, faces):
    arr = (ctypes.c_int32 * 6)(*[int(bool(f)) for f in faces])
    _check(lib().fsi_pressure_set_faces(mesh.handle, arr))


def fsi_pressure_level_sizes(mesh: Mesh):
    """Unknowns per level of the pressure hierarchy (either mesh kind)."""
    n = ctypes.c_int32(0)
    buf = (ctypes.c_int64 * 16)()
    _check(lib().fsi_pressure_level_sizes(mesh.handle, ctypes.byref(n), buf))
    return [int(buf[l]) for l in range(n.value)]


def fsi_pressure_use_amg(mesh: Mesh, on=True):
    """Structured grid: pressure block from the algebraic multigrid of the
    assembled Q1 element matrices (on) or the geometric multigrid (off)."""
    _check(lib().fsi_pressure_use_amg(mesh.handle, int(bool(on))))


def fsi_pressure_set_eliminated(mesh: Mesh, eliminated=None):
    """Algebraic multigrid (tetrahedral mesh or fsi_pressure_use_amg):
    per-node uint8 device flags of eliminated pressure nodes (None: none)."""
    if eliminated is None:
        _check(lib().fsi_pressure_set_eliminated(mesh.handle, None))
        return
    import torch
    if eliminated.dtype != torch.uint8 or eliminated.numel() != mesh.n_nodes:
        raise ValueError("eliminated must be a uint8 tensor of n_nodes entries")
    _check(lib().fsi_pressure_set_eliminated(mesh.handle, _ptr(eliminated.contiguous())))


def fsi_pressure_apply(mesh: Mesh, level, x, y):
    p = _prec_of(x)
    dt = _prec_dtype(p)
    _check(lib().fsi_pressure_apply(mesh.handle, p, int(level), _ptr(x, dt), _ptr(y, dt)))


def fsi_pressure_restrict(mesh: Mesh, level, r, b):
    p = _prec_of(r)
    dt = _prec_dtype(p)
    _check(lib().fsi_pressure_restrict(mesh.handle, p, int(level), _ptr(r, dt), _ptr(b, dt)))


def fsi_pressure_prolong_add(mesh: Mesh, level, xc, x):
    p = _prec_of(x)
    dt = _prec_dtype(p)
    _check(lib().fsi_pressure_prolong_add(mesh.handle, p, int(level), _ptr(xc, dt), _ptr(x, dt)))


def fsi_pressure_smooth(mesh: Mesh, level, degree, b, x, from_zero=True):
    p = _prec_of(x)
    dt = _prec_dtype(p)
    _check(lib().fsi_pressure_smooth(mesh.handle, p, int(level), int(degree), _ptr(b, dt),
                                     _ptr(x, dt), 1 if from_zero else 0))


def fsi_pressure_vcycle(mesh: Mesh, b, x):
    p = _prec_of(x)
    dt = _prec_dtype(p)
    _check(lib().fsi_pressure_vcycle(mesh.handle, p, _ptr(b, dt), _ptr(x, dt)))


class Batch:
    """Owner of an fsi_batch; keeps the meshes and item tensors alive."""

    def __init__(self, meshes, items, prec, stream):
        self.meshes, self.items_t = meshes, items
        arr = (fsi_batch_item * len(items))()
        dt = _prec_dtype(prec)
        import torch
        for i, it in enumerate(items):
            m = 0 if it.get("elem") is None else int(it["elem"].shape[0])
            arr[i] = fsi_batch_item(
                _ptr(it["U"], dt), _ptr(it["A"], dt), _ptr(it.get("f"), dt), _ptr(it["x"], dt),
                _ptr(it["R"], dt), _ptr(it["Jx"], dt), m, _ptr(it.get("elem"), torch.int32),
                _ptr(it["cell_start"], torch.int32), _ptr(it.get("perm"), torch.int32),
                _ptr(it.get("xi"), dt), _ptr(it.get("lam"), dt), _ptr(it.get("w"), dt),
                _ptr(it.get("u"), dt), _ptr(it["F"], dt), _ptr(it.get("X"), torch.float64))
        handles = (ctypes.c_void_p * len(meshes))(*[mm.handle.value for mm in meshes])
        out = ctypes.c_void_p()
        _check(lib().fsi_batch_create(handles, arr, len(items), prec, ctypes.c_void_p(stream),
                                      ctypes.byref(out)))
        self.handle = out

    def run(self, mode):
        _check(lib().fsi_batch_run(self.handle, mode))

    def time(self, mode, reps=5):
        out = ctypes.c_double(0.0)
        _check(lib().fsi_batch_time(self.handle, mode, reps, ctypes.byref(out)))
        return out.value

    def autotune(self, reps=3):
        r = fsi_tune_report()
        _check(lib().fsi_batch_autotune(self.handle, reps, ctypes.byref(r)))
        cands = [(r.cand_bx[i], r.cand_by[i], r.cand_bz[i], r.cand_ctas[i], r.cand_seconds[i])
                 for i in range(r.n_candidates)]
        return {"brick": (r.bx, r.by, r.bz), "threads": r.threads, "ctas_per_sm": r.ctas_per_sm,
                "seconds": r.seconds, "candidates": cands}

    def close(self):
        if getattr(self, "handle", None):
            lib().fsi_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fsi_mesh_set_brick(mesh: Mesh, op, prec, bx, by, bz, threads):
    _check(lib().fsi_mesh_set_brick(mesh.handle, op, prec, bx, by, bz, threads))


def fsi_mesh_autotune(mesh: Mesh, op, prec, reps=5):
    """Time the candidate brick shapes of one VMS operator (0 residual, 1
    Jacobian) in `prec` and keep the fastest; returns the choice and the
    per-candidate seconds per launch."""
    r = fsi_tune_report()
    _check(lib().fsi_mesh_autotune(mesh.handle, int(op), int(prec), int(reps), ctypes.byref(r)))
    cands = [((r.cand_bx[i], r.cand_by[i], r.cand_bz[i]), r.cand_ctas[i], r.cand_seconds[i])
             for i in range(r.n_candidates)]
    return {"brick": (r.bx, r.by, r.bz), "threads": r.threads, "seconds": r.seconds,
            "candidates": cands}
