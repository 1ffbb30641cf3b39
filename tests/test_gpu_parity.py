"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on
the same seeded inputs.

Tolerances: 1e-12 in FP64 and double-float, 1e-5 in FP32 (FP32 inputs rounded
from the FP64 data; the oracle runs in FP64 on the rounded values), held by
every part of an output (tests/parity.py): the momentum and continuity rows
apart, the boundary and interior nodes apart, norm-wise and for the largest
entry error.  Location indices and the cell
table are compared bit for bit.
"""
import numpy as np
import pytest

import parity

from paper_2601_08266_gb300 import inputs

pytestmark = pytest.mark.gpu

# Double-float (FSI_DF64) keeps ~48 significand bits and its additions are
# accurate relative to the larger operand (2^-47 against FP64's 2^-53), so on
# a part of an output whose value is a cancellation of larger terms its error
# is up to 2^6 = 64 times native FP64's.  The worst part of the 128^3
# workload (the residual's continuity row) carries 5.3e-14 in native FP64;
# 64 x 5.3e-14 = 3.4e-12, and the bar keeps a factor ~3 above that.
TOL_DF64 = 1e-11
TOL = {"f64": 1e-12, "f32": 1e-5, "df64": TOL_DF64}


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
    """Round FP64 data to the working precision and back (the oracle's input)."""
    return a.astype(np.float32).astype(np.float64) if prec == "f32" else a


def dtype_of(prec):
    import torch
    return torch.float32 if prec == "f32" else torch.float64


def make(fsi, oracle, N, h=None, x0=(0.0, 0.0, 0.0), **phys):
    p = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, has_s=False)
    p.update(phys)
    mesh = fsi.Mesh(N, x0=x0, h=h, **p, device=0)
    grid = oracle.core.Grid(N, x0=x0, h=h)
    return mesh, grid, p


def vms_case(fsi, oracle, mesh, grid, p, U, A, f, x, prec):
    import torch
    P = {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]
    dt = dtype_of(prec)
    U, A, x = cast(prec, U), cast(prec, A), cast(prec, x)
    f = None if f is None else cast(prec, f)
    Ud, Ad, xd = T(U, dt), T(A, dt), T(x, dt)
    fd = None if f is None else T(f, dt)
    R = torch.empty_like(Ud)
    Jx = torch.empty_like(Ud)
    fsi.fsi_residual(mesh, P, Ud, Ad, fd, R)
    fsi.fsi_jacobian_apply(mesh, P, Ud, Ad, fd, xd, Jx)
    torch.cuda.synchronize()
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    Ro = oracle.core.residual(grid, p, U, A, f=f)
    Jo = oracle.core.jacobian_apply(grid, p, U, A, x, c_a, c_v, f=f)
    return rel(H(R), Ro, grid.N), rel(H(Jx), Jo, grid.N), (R, Jx)


# ---------------------------------------------------------------- stage
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_stage_matches_generalized_alpha(fsi, oracle, prec):
    import torch
    mesh, grid, p = make(fsi, oracle, 5, dt=0.013)
    n = mesh.n_nodes
    rng = np.random.default_rng(0)
    y, Vn, An = (cast(prec, rng.normal(size=(n, 4))) for _ in range(3))
    s = cast(prec, rng.uniform(1, 3, n))
    dt = dtype_of(prec)
    P = fsi.FSI_F64 if prec == "f64" else fsi.FSI_F32
    U = torch.empty((n, 4), dtype=dt, device="cuda")
    A = torch.empty_like(U)
    fsi.fsi_stage(mesh, P, T(y, dt), T(Vn, dt), T(An, dt), T(s, dt), U, A)
    Uo, Ao = oracle.timeint.stage(y, Vn, An, p["dt"], p["rho_inf"], s=s)
    assert rel(H(U), Uo) < TOL[prec] and rel(H(A), Ao) < TOL[prec]


# ---------------------------------------------------------------- VMS
@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_vms_config1_one_implicit_step(fsi, oracle, prec):
    """8^3 grid, y ~ U[-1,1], zero history, stage by generalized alpha."""
    mesh, grid, p = make(fsi, oracle, 8)
    y, Vn, An = inputs.uniform_state(8, seed=0)
    U, A = oracle.timeint.stage(y, Vn, An, p["dt"], p["rho_inf"])
    x = inputs.uniform_nodal(8, seed=1)
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, U, A, None, x, prec)
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("N,h", [((13, 10, 9), (0.07, 0.11, 0.09)), ((1, 1, 1), (0.3, 0.3, 0.3)),
                                 ((17, 3, 5), None)])
def test_vms_ragged_bricks_anisotropic(fsi, oracle, prec, N, h):
    """Several bricks with ragged tails, anisotropic cells, s field, body force,
    rho != 1 and O(1) velocities (tau depends on v)."""
    mesh, grid, p = make(fsi, oracle, N, h=h, x0=(0.2, -0.1, 0.4), rho=1.3, mu=0.02,
                         dt=0.01, rho_inf=0.3, has_s=True)
    n = mesh.n_nodes
    rng = np.random.default_rng(sum(N))
    U = rng.uniform(-2, 2, (n, 4))
    A = rng.uniform(-1, 1, (n, 4))
    A[:, 3] = rng.uniform(1.0, 50.0, n)
    f = rng.normal(size=(n, 4))
    x = rng.normal(size=(n, 4))
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, U, A, f, x, prec)
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ


def test_vms_deterministic(fsi, oracle):
    import torch
    mesh, grid, p = make(fsi, oracle, (12, 9, 7))
    n = mesh.n_nodes
    rng = np.random.default_rng(1)
    U, A, x = (T(rng.normal(size=(n, 4))) for _ in range(3))
    outs = []
    for _ in range(2):
        R = torch.empty_like(U)
        J = torch.empty_like(U)
        fsi.fsi_residual(mesh, fsi.FSI_F64, U, A, None, R)
        fsi.fsi_jacobian_apply(mesh, fsi.FSI_F64, U, A, None, x, J)
        outs.append((R.clone(), J.clone()))
    assert torch.equal(outs[0][0], outs[1][0]) and torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_vms_config2_full_size(fsi, oracle, prec):
    """64^3 grid (262k elements, 1.1M DOFs), smooth Fourier velocity and pressure
    plus noise: the whole residual and Jacobian apply against the oracle."""
    N = 64
    mesh, grid, p = make(fsi, oracle, N)
    U = inputs.fourier_field(N, seed=10)
    A = np.zeros_like(U)
    A[:, :3] = inputs.fourier_field(N, seed=11, ncomp=3)
    A[:, 3] = 1.0
    x = inputs.uniform_nodal(N, seed=12)
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, U, A, None, x, prec)
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ
    print(f"\n64^3 {prec}: residual rel err {eR:.2e}, Jacobian rel err {eJ:.2e}")


# ---------------------------------------------------------------- DLM
def dlm_run(fsi, mesh, X, prec, lam, w, U, F0, accumulate):
    import torch
    dt = dtype_of(prec)
    P = {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]
    m = X.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    nout = fsi.fsi_locate(mesh, T(X), elem, xi, cs, perm)
    xiw = xi.to(dt)
    u = torch.empty((m, 3), dtype=dt, device="cuda")
    fsi.fsi_dlm_interp(mesh, P, elem, xiw, T(U, dt), u)
    F = T(F0, dt).clone()
    fsi.fsi_dlm_spread(mesh, P, elem, xiw, cs, perm, T(lam, dt),
                       None if w is None else T(w, dt), F, accumulate)
    torch.cuda.synchronize()
    return dict(elem=elem.cpu().numpy(), xi=H(xi), cs=cs.cpu().numpy(), perm=perm.cpu().numpy(),
                nout=nout, u=H(u), F=H(F))


def dlm_check(fsi, oracle, N, X, prec, weighted, accumulate, seed=0, h=None, x0=(0, 0, 0)):
    mesh, grid, _ = make(fsi, oracle, N, h=h, x0=x0)
    rng = np.random.default_rng(seed)
    m = X.shape[0]
    lam = cast(prec, rng.normal(size=(m, 3)))
    w = cast(prec, rng.uniform(0.5, 2, m)) if weighted else None
    U = cast(prec, rng.normal(size=(mesh.n_nodes, 4)))
    F0 = cast(prec, rng.normal(size=(mesh.n_nodes, 4)))
    g = dlm_run(fsi, mesh, X, prec, lam, w, U, F0, accumulate)
    eo, xio, nouto = oracle.core.locate(grid, X)
    cso, permo = oracle.core.cell_hash(grid, eo)
    assert g["nout"] == nouto
    assert np.array_equal(g["elem"], eo)
    assert np.array_equal(g["xi"], xio)
    assert np.array_equal(g["cs"], cso)
    assert np.array_equal(g["perm"], permo)
    xiw = cast(prec, xio)
    uo = oracle.core.interp(grid, eo, xiw, U)
    Fo = oracle.core.spread(grid, eo, xiw, lam, w=w, F=F0, accumulate=accumulate)
    assert rel(g["u"], uo) < TOL[prec]
    assert rel(g["F"][:, :3], Fo[:, :3], grid.N) < TOL[prec]
    # slot 3 is never written
    assert np.array_equal(g["F"][:, 3], F0[:, 3].astype(np.float32).astype(np.float64)
                          if prec == "f32" else F0[:, 3])
    return g


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("weighted,accumulate", [(False, False), (True, True)])
def test_dlm_config1_ball(fsi, oracle, prec, weighted, accumulate):
    X = inputs.ball_points(500, seed=2)
    dlm_check(fsi, oracle, 8, X, prec, weighted, accumulate)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_dlm_edges_outside_and_boundaries(fsi, oracle, prec):
    X = inputs.edge_points((6, 5, 7), seed=4, m_random=3000)
    X = X * np.array([1.2, 0.5, 0.7])
    g = dlm_check(fsi, oracle, (6, 5, 7), X, prec, True, True, h=(0.2, 0.1, 0.1))
    assert g["nout"] > 0


def test_dlm_empty_and_all_outside(fsi, oracle):
    import torch
    mesh, grid, _ = make(fsi, oracle, 4)
    for X in (np.zeros((0, 3)), np.full((37, 3), 5.0)):
        m = X.shape[0]
        lam = np.ones((m, 3))
        U = np.ones((mesh.n_nodes, 4))
        F0 = np.full((mesh.n_nodes, 4), 2.0)
        g = dlm_run(fsi, mesh, X, "f64", lam, None, U, F0, True)
        assert g["nout"] == m
        assert np.all(g["cs"] == 0)
        assert np.array_equal(g["perm"], np.arange(m))
        assert np.all(g["u"] == 0) and np.array_equal(g["F"], F0)
        g = dlm_run(fsi, mesh, X, "f64", lam, None, U, F0, False)
        assert np.all(g["F"][:, :3] == 0)


def test_dlm_medium_density_cells(fsi, oracle):
    """33..64 points per cell (one lane's bitonic network), 65..128 (the warp's
    register rank sort) and > 128 (four-lane spreading groups give way to the
    whole warp above 128 points)."""
    X = np.random.default_rng(4).uniform(size=(400, 3))
    dlm_check(fsi, oracle, 2, X, "f64", True, False)
    dlm_check(fsi, oracle, 2, X, "df64", False, True)
    X = np.random.default_rng(5).uniform(size=(700, 3))
    dlm_check(fsi, oracle, 2, X, "f64", True, False)
    dlm_check(fsi, oracle, 2, X, "df64", True, True)
    X = np.random.default_rng(6).uniform(size=(1500, 3))
    dlm_check(fsi, oracle, 2, X, "f64", False, True)


def test_dlm_dense_cell_and_strict(fsi, oracle):
    """Many points in one cell (the long-slice sort path) and strict mode."""
    import torch
    rng = np.random.default_rng(3)
    X = 0.1 + 0.05 * rng.uniform(size=(5000, 3))
    X = np.concatenate([X, rng.uniform(size=(300, 3))])
    dlm_check(fsi, oracle, 4, X, "f64", False, False)
    mesh, _, _ = make(fsi, oracle, 4)
    elem = torch.empty(2, dtype=torch.int32, device="cuda")
    xi = torch.empty((2, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fsi.FsiError) as ei:
        fsi.fsi_locate(mesh, T(np.array([[0.5, 0.5, 0.5], [2.0, 0.5, 0.5]])), elem, xi,
                       strict=True)
    assert ei.value.status == 4


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_dlm_config2_leaflets_full_size(fsi, oracle, prec):
    """64^3 grid, 200k points on three thin leaflets (all inside)."""
    X = inputs.leaflet_points(200_000, seed=20)
    g = dlm_check(fsi, oracle, 64, X, prec, False, True)
    assert g["nout"] == 0


@pytest.mark.parametrize("layers", [0, 1, 2])
def test_interface_scaling_matches_oracle(fsi, oracle, layers):
    """Sec. 2.1's band field from located leaflet points, bit-exact, and a
    VMS residual on a mesh with has_s that uses it."""
    import torch
    from oracle import interface as itf
    N = (20, 16, 18)
    mesh, grid, p = make(fsi, oracle, N, has_s=True)
    X = inputs.leaflet_points(3000, seed=31)
    m = X.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    fsi.fsi_locate(mesh, T(X), elem, xi, cs, perm)
    s = torch.empty(mesh.n_nodes, dtype=torch.float64, device="cuda")
    fsi.fsi_interface_scaling(mesh, cs, 100.0, layers, s)
    torch.cuda.synchronize()
    e, _, _ = oracle.core.locate(grid, X)
    ref = itf.scaling_field(grid, e, 100.0, layers)
    assert np.array_equal(H(s), ref)
    assert (ref == 100.0).sum() > 0 and (ref == 1.0).sum() > 0
    # the field in the acceleration's 4th slot scales tau_M in the VMS operators
    rng = np.random.default_rng(layers)
    U = rng.uniform(-1, 1, (mesh.n_nodes, 4))
    A = rng.uniform(-1, 1, (mesh.n_nodes, 4))
    A[:, 3] = ref
    x = rng.uniform(-1, 1, (mesh.n_nodes, 4))
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, U, A, None, x, "df64")
    assert eR < TOL_DF64 and eJ < TOL_DF64


# ---------------------------------------------------------------- full sizes
_C3 = {}


def config3_inputs():
    """128^3 channel-like state (8.6 M DOFs): inflow profile
    v_x = 16 y(1-y) z(1-z) plus 0.01 x a seeded Fourier field, Fourier
    pressure, acceleration and direction; 1 M points on three leaflets."""
    if not _C3:
        N = 128
        ax = np.arange(N + 1) / N
        z, y, _ = np.meshgrid(ax, ax, ax, indexing="ij")
        U = 0.01 * inputs.fourier_field(N, seed=40)
        U[:, 0] += (16.0 * y * (1 - y) * z * (1 - z)).ravel()
        A = np.zeros_like(U)
        A[:, :3] = inputs.fourier_field(N, seed=41, ncomp=3)
        A[:, 3] = 1.0
        _C3.update(N=N, U=U, A=A, x=inputs.uniform_nodal(N, seed=42),
                   X=inputs.leaflet_points(1_000_000, seed=43))
    return _C3


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_vms_config3_full_size(fsi, oracle, prec):
    """128^3 grid (2.1 M elements, 8.6 M DOFs, mu = 1e-3): the whole residual
    and Jacobian apply against the oracle, part by part (32-bit index
    products of the brick and gather kernels are largest here)."""
    W = config3_inputs()
    mesh, grid, p = make(fsi, oracle, W["N"], mu=1e-3)
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, W["U"], W["A"], None, W["x"], prec)
    print(f"\n128^3 {prec}: residual {eR:.2e}, Jacobian {eJ:.2e}")
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ
    mesh.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_dlm_config3_full_size(fsi, oracle, prec):
    """128^3 grid, 1 M leaflet points: location and cell table bit for bit,
    interpolation and weighted accumulating spreading part by part."""
    W = config3_inputs()
    g = dlm_check(fsi, oracle, W["N"], W["X"], prec, True, True, seed=44)
    assert g["nout"] == 0


def test_fused_config3_full_size(fsi, oracle):
    """The fused residual + Jacobian pass of the benchmark step at 128^3 in
    native FP64 and double-float against the oracle."""
    import torch
    W = config3_inputs()
    mesh, grid, p = make(fsi, oracle, W["N"], mu=1e-3)
    Ud, Ad, xd = T(W["U"]), T(W["A"]), T(W["x"])
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    Ro = oracle.core.residual(grid, p, W["U"], W["A"])
    Jo = oracle.core.jacobian_apply(grid, p, W["U"], W["A"], W["x"], c_a, c_v)
    for P in (fsi.FSI_F64, fsi.FSI_DF64):
        R = torch.empty_like(Ud)
        J = torch.empty_like(Ud)
        fsi.fsi_residual_jacobian_apply(mesh, P, Ud, Ad, None, xd, R, J)
        torch.cuda.synchronize()
        tol = TOL["f64"] if P == fsi.FSI_F64 else TOL_DF64
        assert rel(H(R), Ro, grid.N) < tol and rel(H(J), Jo, grid.N) < tol
    mesh.close()


@pytest.mark.parametrize("prec", ["f64", "df64", "f32"])
def test_vms_paper_scales(fsi, oracle, prec):
    """Inputs at the scales of the paper's problems (CGS units): element size
    1e-3 cm, time step 1e-5 s (free-falling sphere), blood-like viscosity
    0.035 P, velocities up to 100 cm/s, accelerations up to 1e6 cm/s^2 and a
    pressure of 3e5 dyn/cm^2 with +-10 % variation (closed valve).  tau_M is
    ~6e-7 here and the metric G ~ 4e6, far from the unit scales of the other
    cases; double-float must still hold its bar."""
    N, h = (20, 14, 23), (1e-3, 1e-3, 1e-3)
    mesh, grid, p = make(fsi, oracle, N, h=h, x0=(0.51, -0.013, 0.2), rho=1.06, mu=0.035,
                         dt=1e-5, has_s=True)
    n = mesh.n_nodes
    rng = np.random.default_rng(77)
    U = np.empty((n, 4))
    U[:, :3] = rng.uniform(-100.0, 100.0, (n, 3))
    U[:, 3] = 3e5 * (1.0 + rng.uniform(-0.1, 0.1, n))
    A = np.empty((n, 4))
    A[:, :3] = rng.uniform(-1e6, 1e6, (n, 3))
    A[:, 3] = rng.uniform(1.0, 100.0, n)
    f = np.zeros((n, 4))
    f[:, 2] = -981.0
    x = np.empty((n, 4))
    x[:, :3] = rng.uniform(-1e6, 1e6, (n, 3))
    x[:, 3] = rng.uniform(-3e4, 3e4, n)
    eR, eJ, _ = vms_case(fsi, oracle, mesh, grid, p, U, A, f, x, prec)
    print(f"\npaper scales {prec}: residual {eR:.2e}, Jacobian {eJ:.2e}")
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ


def test_dlm_paper_scales(fsi, oracle):
    """Location, interpolation and spreading on a 1e-3 cm grid away from the
    origin (x0 ~ 0.5 cm: t = (X - x0)/h loses ~10 bits to the offset),
    velocities ~100 cm/s and multipliers ~1e5: FP64 and double-float against
    the oracle."""
    N, h, x0 = (30, 24, 28), (1e-3,) * 3, (0.5, 0.25, -0.75)
    rng = np.random.default_rng(5)
    X = np.array(x0) + rng.uniform(-0.001, 1.001, (20_000, 3)) * np.array(N) * 1e-3
    for prec in ("f64", "df64"):
        mesh, grid, _ = make(fsi, oracle, N, h=h, x0=x0)
        m = X.shape[0]
        lam = 1e5 * rng.normal(size=(m, 3))
        U = 100.0 * rng.normal(size=(mesh.n_nodes, 4))
        g = dlm_run(fsi, mesh, X, prec, lam, None, U, np.zeros((mesh.n_nodes, 4)), False)
        eo, xio, nouto = oracle.core.locate(grid, X)
        assert g["nout"] == nouto and np.array_equal(g["elem"], eo)
        assert np.array_equal(g["xi"], xio)
        assert rel(g["u"], oracle.core.interp(grid, eo, xio, U)) < TOL[prec]
        Fo = oracle.core.spread(grid, eo, xio, lam)
        assert rel(g["F"][:, :3], Fo[:, :3], grid.N) < TOL[prec]
