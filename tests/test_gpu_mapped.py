"""GPU parity on mapped (curvilinear) structured grids: VMS residual and
Jacobian apply with per-Gauss-point geometry from the trilinear map, point
location by the element walk with Newton inversion, interpolation/spreading
on the located points and the Newton step, against the oracle's mapped-grid
operators (node coordinates given to both sides)."""
import numpy as np
import pytest

import parity

from paper_2601_08266_gb300 import inputs

pytestmark = pytest.mark.gpu

# double-float's bar (its additions are accurate to 2^-47 of the larger
# operand, 64 x FP64's unit roundoff; see test_gpu_parity.py)
TOL = {"f64": 1e-12, "f32": 1e-5, "df64": 1e-11}


@pytest.fixture(scope="module")
def fsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08266_gb300 as pkg
    return pkg


def T(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    return t.to(dtype) if dtype is not None else t


def H(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b, grid=None):
    """Worst local relative error of a against b: momentum and continuity
    rows, boundary and interior nodes (when grid is given) apart, norm-wise
    and largest entry (tests/parity.py)."""
    return parity.rel_local(np.asarray(a), b, grid)


def rel_norm(a, b):
    """Norm-wise distance of a whole solution vector from a reference one."""
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - b) / (nb if nb > 0 else 1.0)


def cast(prec, a):
    return a.astype(np.float32).astype(np.float64) if prec == "f32" else a


def dtype_of(prec):
    import torch
    return torch.float32 if prec == "f32" else torch.float64


def distorted(core, N, x0=(0.0, 0.0, 0.0), h=None, amp=0.15, seed=0, interior_only=False):
    """Node coordinates of the nominal grid moved by up to amp * h per axis
    (non-affine hexahedra with positive Jacobians)."""
    g = core.Grid(N, x0=x0, h=h)
    X = g.node_coords()
    rng = np.random.default_rng(seed)
    d = amp * rng.uniform(-1, 1, X.shape) * np.asarray(g.h)[None, :]
    if interior_only:
        lo, hi = np.asarray(x0), np.asarray(x0) + np.asarray(g.N) * np.asarray(g.h)
        d[np.any((X < lo + 1e-12) | (X > hi - 1e-12), axis=1)] = 0.0
    return X + d


def bubble(X, delta):
    b = np.sin(2 * np.pi * X[:, 0]) * np.sin(2 * np.pi * X[:, 1]) * np.sin(2 * np.pi * X[:, 2])
    return X + delta * b[:, None] * np.array([1.0, -0.7, 0.4])[None, :]


def mapped_mesh(fsi, N, X, x0=(0.0, 0.0, 0.0), h=None, **phys):
    p = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, has_s=False)
    p.update(phys)
    mesh = fsi.Mesh(N, x0=x0, h=h, **p, device=0)
    mesh.set_coordinates(T(X))
    return mesh, p


def vms(fsi, mesh, prec, U, A, f, x):
    import torch
    P = {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]
    dt = dtype_of(prec)
    Ud, Ad, xd = T(U, dt), T(A, dt), T(x, dt)
    fd = None if f is None else T(f, dt)
    R, Jx = torch.empty_like(Ud), torch.empty_like(Ud)
    fsi.fsi_residual(mesh, P, Ud, Ad, fd, R)
    fsi.fsi_jacobian_apply(mesh, P, Ud, Ad, fd, xd, Jx)
    torch.cuda.synchronize()
    return H(R), H(Jx)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("N,h", [((13, 10, 9), (0.07, 0.11, 0.09)), ((1, 1, 1), (0.3, 0.3, 0.3)),
                                 ((17, 3, 5), None)])
def test_mapped_vms_ragged_bricks(fsi, oracle, prec, N, h):
    """Distorted hexahedra over several bricks with ragged tails, s field,
    body force and O(1) velocities."""
    core = oracle.core
    x0 = (0.2, -0.1, 0.4)
    X = distorted(core, N, x0=x0, h=h, seed=sum(N))
    mesh, p = mapped_mesh(fsi, N, X, x0=x0, h=h, rho=1.3, mu=0.02, dt=0.01, rho_inf=0.3,
                          has_s=True)
    n = mesh.n_nodes
    rng = np.random.default_rng(sum(N) + 1)
    U = rng.uniform(-2, 2, (n, 4))
    A = rng.uniform(-1, 1, (n, 4))
    A[:, 3] = rng.uniform(1.0, 50.0, n)
    f, x = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    U, A, f, x = (cast(prec, a) for a in (U, A, f, x))
    # the FP32 path stores FP32 node coordinates: the oracle gets them rounded too
    grid = core.Grid(N, coords=cast(prec, X))
    R, Jx = vms(fsi, mesh, prec, U, A, f, x)
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    eR = rel(R, core.residual(grid, p, U, A, f=f), grid.N)
    eJ = rel(Jx, core.jacobian_apply(grid, p, U, A, x, c_a, c_v, f=f), grid.N)
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_mapped_vms_smooth_map_24cubed(fsi, oracle, prec):
    """A smooth bubble map of the unit cube, 24^3 elements, smooth fields."""
    core = oracle.core
    N = 24
    X = bubble(core.Grid(N).node_coords(), 0.03)
    mesh, p = mapped_mesh(fsi, N, X)
    U = inputs.fourier_field(N, seed=20)
    A = np.zeros_like(U)
    A[:, :3] = inputs.fourier_field(N, seed=21, ncomp=3)
    A[:, 3] = 1.0
    x = inputs.uniform_nodal(N, seed=22)
    U, A, x = (cast(prec, a) for a in (U, A, x))
    grid = core.Grid(N, coords=cast(prec, X))
    R, Jx = vms(fsi, mesh, prec, U, A, None, x)
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    eR = rel(R, core.residual(grid, p, U, A), grid.N)
    eJ = rel(Jx, core.jacobian_apply(grid, p, U, A, x, c_a, c_v), grid.N)
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ


def test_uniform_coordinates_reproduce_the_uniform_kernels(fsi, oracle):
    """The mapped path fed the uniform grid's own nodes agrees with the uniform
    path; returning to the uniform grid (NULL coordinates) restores it exactly."""
    core = oracle.core
    N, h, x0 = (9, 7, 6), (0.1, 0.13, 0.08), (0.3, 0.1, -0.2)
    grid = core.Grid(N, x0=x0, h=h)
    mesh, p = mapped_mesh(fsi, N, grid.node_coords(), x0=x0, h=h, has_s=True, dt=0.02)
    n = mesh.n_nodes
    rng = np.random.default_rng(5)
    U, A, f, x = (rng.normal(size=(n, 4)) for _ in range(4))
    A[:, 3] = rng.uniform(1, 3, n)
    Rm, Jm = vms(fsi, mesh, "f64", U, A, f, x)
    mesh.set_coordinates(None)
    Ru, Ju = vms(fsi, mesh, "f64", U, A, f, x)
    assert rel(Rm, Ru) < 1e-13 and rel(Jm, Ju) < 1e-13
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    assert np.array_equal(Ru, vms(fsi, mesh, "f64", U, A, f, x)[0])
    assert rel(Ru, core.residual(grid, p, U, A, f=f)) < 1e-12
    assert rel(Ju, core.jacobian_apply(grid, p, U, A, x, c_a, c_v, f=f)) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_geometry_follows_new_coordinates_and_physics(fsi, oracle, prec):
    """The per-Gauss-point geometry table is rebuilt when the coordinates
    change and stays valid when only the physics changes."""
    core = oracle.core
    N = (6, 5, 7)
    X1 = distorted(core, N, seed=31)
    X2 = distorted(core, N, seed=32, amp=0.2)
    mesh, p = mapped_mesh(fsi, N, X1, has_s=True)
    n = mesh.n_nodes
    rng = np.random.default_rng(33)
    U, A, x = (cast(prec, rng.normal(size=(n, 4))) for _ in range(3))
    A[:, 3] = cast(prec, rng.uniform(1.0, 3.0, n))
    for X, phys in ((X1, {}), (X2, {}), (X2, dict(mu=0.05, dt=0.02)), (X1, dict(mu=0.05, dt=0.02))):
        if phys:
            mesh.set_physics(**phys)
            p.update(phys)
        mesh.set_coordinates(T(X))
        grid = core.Grid(N, coords=cast(prec, X))
        R, Jx = vms(fsi, mesh, prec, U, A, None, x)
        c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
        assert rel(R, core.residual(grid, p, U, A), grid.N) < TOL[prec]
        assert rel(Jx, core.jacobian_apply(grid, p, U, A, x, c_a, c_v), grid.N) < TOL[prec]


def element_nodes(N, e):
    ex, ey, ez = e % N[0], (e // N[0]) % N[1], e // (N[0] * N[1])
    return [(ex + (a & 1)) + (N[0] + 1) * ((ey + ((a >> 1) & 1)) + (N[1] + 1) * (ez + ((a >> 2) & 1)))
            for a in range(8)]


def map_points(core, grid, X, e, xi):
    P = np.zeros((len(e), 3))
    for b in range(len(e)):
        Nv, _ = core.shape(xi[b])
        P[b] = Nv @ X[element_nodes(grid.N, e[b])]
    return P


def points_in_elements(core, grid, X, m, seed, lo=-0.95, hi=0.95):
    """Points mapped from random (element, xi): the true element is unique."""
    rng = np.random.default_rng(seed)
    e = rng.integers(0, grid.n_elems, m)
    xi = rng.uniform(lo, hi, (m, 3))
    return map_points(core, grid, X, e, xi), e.astype(np.int32), xi


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_mapped_locate_interp_spread(fsi, oracle, prec):
    import torch
    core = oracle.core
    N = (7, 6, 5)
    X = distorted(core, N, seed=3, amp=0.2, interior_only=True)
    grid = core.Grid(N, coords=X)
    mesh, _ = mapped_mesh(fsi, N, X)
    P, e_true, xi_true = points_in_elements(core, grid, X, 800, seed=4)
    P = np.concatenate([P, [[1.5, 0.5, 0.5], [-0.1, 0.2, 0.3], [0.5, 0.5, 2.0]]])
    m = P.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    nout = fsi.fsi_locate(mesh, T(P), elem, xi, cs, perm)
    eo, xio, nouto = core.locate(grid, P)
    assert nout == nouto == 3
    eg = elem.cpu().numpy()
    assert np.array_equal(eg, eo) and np.array_equal(eg[:-3], e_true)
    assert np.abs(H(xi) - xio).max() < 1e-12
    cso, permo = core.cell_hash(grid, eo)
    assert np.array_equal(cs.cpu().numpy(), cso) and np.array_equal(perm.cpu().numpy(), permo)
    rng = np.random.default_rng(6)
    dt = dtype_of(prec)
    Pp = {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]
    U = cast(prec, rng.normal(size=(mesh.n_nodes, 4)))
    lam = cast(prec, rng.normal(size=(m, 3)))
    w = cast(prec, rng.uniform(0.5, 2, m))
    u = torch.empty((m, 3), dtype=dt, device="cuda")
    xiw = xi.to(dt)
    fsi.fsi_dlm_interp(mesh, Pp, elem, xiw, T(U, dt), u)
    F = torch.zeros((mesh.n_nodes, 4), dtype=dt, device="cuda")
    fsi.fsi_dlm_spread(mesh, Pp, elem, xiw, cs, perm, T(lam, dt), T(w, dt), F, False)
    torch.cuda.synchronize()
    xw = cast(prec, H(xi))
    assert rel(H(u), core.interp(grid, eo, xw, U)) < TOL[prec]
    assert rel(H(F)[:, :3], core.spread(grid, eo, xw, lam, w=w)[:, :3], grid.N) < TOL[prec]


@pytest.mark.parametrize("delta", [0.03, 0.08])
def test_mapped_locate_walks_across_elements(fsi, oracle, delta):
    """A smooth map that moves nodes by up to 1 and 2.6 element widths: the
    nominal start element is far off and the walk has to travel; every point
    mapped from (element, xi) is found there with that xi."""
    import torch
    core = oracle.core
    N = 32
    X = bubble(core.Grid(N).node_coords(), delta)
    grid = core.Grid(N, coords=X)
    mesh, _ = mapped_mesh(fsi, N, X)
    P, e_true, xi_true = points_in_elements(core, grid, X, 4000, seed=15, lo=-0.999, hi=0.999)
    m = P.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    nout = fsi.fsi_locate(mesh, T(P), elem, xi)
    assert nout == 0
    assert np.array_equal(elem.cpu().numpy(), e_true)
    assert np.abs(H(xi) - xi_true).max() < 1e-12


def test_mapped_locate_faces_and_nodes_are_valid(fsi, oracle):
    """Points on element faces and at nodes belong to several elements: the
    walk's answer must be one of them (|xi| <= 1 + 1e-10, maps back to X)."""
    import torch
    core = oracle.core
    N = (5, 5, 4)
    X = distorted(core, N, seed=8, amp=0.2, interior_only=True)
    grid = core.Grid(N, coords=X)
    mesh, _ = mapped_mesh(fsi, N, X)
    rng = np.random.default_rng(10)
    P1, _, _ = points_in_elements(core, grid, X, 300, seed=9, lo=-1.0, hi=1.0)
    # one xi component snapped to a face, and points on edges (two snapped)
    e2 = rng.integers(0, grid.n_elems, 400)
    xi2 = rng.uniform(-1, 1, (400, 3))
    xi2[np.arange(400), rng.integers(0, 3, 400)] = rng.choice([-1.0, 1.0], 400)
    xi2[:100, (np.arange(100) + 1) % 3] = 1.0
    P2 = map_points(core, grid, X, e2, xi2)
    P = np.concatenate([P1, X[rng.integers(0, len(X), 100)], P2])
    m = P.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    nout = fsi.fsi_locate(mesh, T(P), elem, xi, cs, perm)
    assert nout == 0
    eg, xg = elem.cpu().numpy(), H(xi)
    assert np.all(np.abs(xg) <= 1 + 1e-10)
    assert np.all((eg >= 0) & (eg < grid.n_elems))
    assert np.abs(map_points(core, grid, X, eg, xg) - P).max() < 1e-12


@pytest.mark.parametrize("mixed,amg", [(False, False), (True, False), (True, True)])
def test_mapped_newton_step(fsi, oracle, mixed, amg):
    """The implicit step on a mapped grid with immersed points: the GPU Newton
    step reaches ||R|| <= 1e-8 ||R0|| by the oracle's mapped-grid residual and
    lands on the oracle's direct-solve solution."""
    import torch
    from oracle import newton
    core = oracle.core
    N = 8
    X = distorted(core, N, seed=12, amp=0.15, interior_only=True)
    grid = core.Grid(N, coords=X)
    n = grid.n_nodes
    rng = np.random.default_rng(13)
    phys = dict(rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, has_s=True)
    Vn, An = 0.5 * rng.normal(size=(n, 4)), 0.5 * rng.normal(size=(n, 4))
    s = rng.uniform(1.0, 3.0, n)
    f = rng.normal(size=(n, 4))
    m = 300
    Pts = inputs.ball_points(m, seed=14, radius=0.3)
    elem, xi, _ = core.locate(grid, Pts)
    w = rng.uniform(0.5, 1.5, m)
    bnd = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    mask = np.zeros((n, 4), dtype=bool)
    mask[bnd, :3] = True
    mask[0, 3] = True
    yD = np.zeros((n, 4))
    yD[bnd, :3] = 0.3 * rng.normal(size=(bnd.sum(), 3))
    solid = dict(drho=0.7, k=2.0, g=(0.0, 0.0, -9.81))
    Pb = newton.Problem(grid, phys, Vn, An, f=f, s=s, mask=mask, yD=yD, points=(elem, xi, w),
                        solid=solid)
    y0 = rng.normal(size=(n, 4))
    y0[mask] = yD[mask]
    mesh, _ = mapped_mesh(fsi, N, X, rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, has_s=True)
    if amg:  # the Schur preconditioner's pressure block assembled on the mapped grid
        fsi.fsi_pressure_use_amg(mesh, True)
    e_d = torch.empty(m, dtype=torch.int32, device="cuda")
    xi_d = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs_d = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    pm_d = torch.empty(m, dtype=torch.int32, device="cuda")
    assert fsi.fsi_locate(mesh, T(Pts), e_d, xi_d, cs_d, pm_d) == 0
    assert np.array_equal(e_d.cpu().numpy(), elem)
    yd = T(y0)
    st = fsi.StepState(yd, T(Vn), T(An), s=T(s), f=T(f), mask=T(mask.astype(np.uint8)),
                       yD=T(yD), elem=e_d, xi=xi_d, cell_start=cs_d, perm=pm_d, w=T(w),
                       drho_s=0.7, k_s=2.0, g_s=(0.0, 0.0, -9.81))
    R = torch.empty_like(yd)
    fsi.fsi_coupled_residual(mesh, st, R)
    torch.cuda.synchronize()
    assert rel(H(R), Pb.residual(y0)) < 1e-12
    code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=12,
                                    max_krylov=2000, newton_rtol=1e-8, krylov_rtol=1e-3)
    assert code == 0 and rep["converged"] == 1, rep
    y_gpu = H(yd)
    assert np.linalg.norm(Pb.residual(y_gpu)) <= 1.01e-8 * rep["r_ref"]
    y_ref, _ = newton.newton(Pb, y0, rtol=1e-13)
    assert rel_norm(y_gpu, y_ref) < 5e-5, rep
