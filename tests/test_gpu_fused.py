"""The fused residual + Jacobian apply (fsi_residual_jacobian_apply): both
operators from one evaluation of the stage per Gauss point.  In double-float
the outputs are bitwise those of the separate calls under the same brick
schedule; in FP64 and FP32 they
agree to rounding; both match the oracle (uniform and mapped grids, ragged
bricks, several brick schedules, s and f present)."""
import numpy as np
import pytest

import parity

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


def run(fsi, mesh, prec, U, A, f, x):
    import torch
    P = {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]
    dt = torch.float32 if prec == "f32" else torch.float64
    Ud, Ad, xd = T(U, dt), T(A, dt), T(x, dt)
    fd = None if f is None else T(f, dt)
    R1, J1, R2, J2 = (torch.empty_like(Ud) for _ in range(4))
    fsi.fsi_residual(mesh, P, Ud, Ad, fd, R1)
    fsi.fsi_jacobian_apply(mesh, P, Ud, Ad, fd, xd, J1)
    fsi.fsi_residual_jacobian_apply(mesh, P, Ud, Ad, fd, xd, R2, J2)
    torch.cuda.synchronize()
    return R1, J1, R2, J2


def inputs_for(n, seed, prec):
    rng = np.random.default_rng(seed)
    U = rng.uniform(-2, 2, (n, 4))
    A = rng.uniform(-1, 1, (n, 4))
    A[:, 3] = rng.uniform(1.0, 30.0, n)
    f, x = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    return tuple(cast(prec, a) for a in (U, A, f, x))


@pytest.mark.parametrize("prec", ["df64", "f64", "f32"])
@pytest.mark.parametrize("mapped", [False, True])
def test_fused_equals_separate_and_oracle(fsi, oracle, prec, mapped):
    import torch
    core = oracle.core
    N, h, x0 = (13, 10, 9), (0.07, 0.11, 0.09), (0.2, -0.1, 0.4)
    p = dict(rho=1.3, mu=0.02, dt=0.01, rho_inf=0.3, has_s=True)
    mesh = fsi.Mesh(N, x0=x0, h=h, **p, device=0)
    grid = core.Grid(N, x0=x0, h=h)
    if mapped:
        X = grid.node_coords()
        rng = np.random.default_rng(7)
        X = X + 0.15 * rng.uniform(-1, 1, X.shape) * np.asarray(h)[None, :]
        mesh.set_coordinates(T(X))
        grid = core.Grid(N, coords=cast(prec, X))
    U, A, f, x = inputs_for(mesh.n_nodes, 11, prec)
    # the element-to-node sums follow the bricks: the same schedule for all three
    slot = {"f32": fsi.FSI_F32, "f64": fsi.FSI_F64, "df64": fsi.FSI_DF64}[prec]
    for op in (0, 1, 2):
        fsi.fsi_mesh_set_brick(mesh, op, slot, 8, 4, 4, 256)
    R1, J1, R2, J2 = run(fsi, mesh, prec, U, A, f, x)
    if prec == "df64":
        assert torch.equal(R1, R2) and torch.equal(J1, J2)
    else:
        assert rel(H(R2), H(R1)) < (1e-13 if prec == "f64" else 1e-6)
        assert rel(H(J2), H(J1)) < (1e-13 if prec == "f64" else 1e-6)
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    assert rel(H(R2), core.residual(grid, p, U, A, f=f), grid.N) < TOL[prec]
    assert rel(H(J2), core.jacobian_apply(grid, p, U, A, x, c_a, c_v, f=f), grid.N) < TOL[prec]


def test_fused_brick_schedules_and_autotune(fsi, oracle):
    import torch
    N = (11, 9, 13)
    mesh = fsi.Mesh(N, device=0, has_s=True)
    U, A, f, x = inputs_for(mesh.n_nodes, 3, "df64")
    g = oracle.core.Grid(N)
    phys = dict(rho=1.0, mu=0.01, dt=1e-3, has_s=True)
    c_a, c_v = oracle.timeint.chain_factors(0.5, 1e-3)
    Rref = oracle.core.residual(g, phys, U, A, f=f)
    Jref = oracle.core.jacobian_apply(g, phys, U, A, x, c_a, c_v, f=f)
    for bx, by, bz, th in [(8, 8, 4, 256), (4, 4, 4, 64), (16, 4, 2, 256), (2, 2, 2, 32)]:
        fsi.fsi_mesh_set_brick(mesh, 2, fsi.FSI_DF64, bx, by, bz, th)
        _, _, R2, J2 = run(fsi, mesh, "df64", U, A, f, x)
        assert rel(H(R2), Rref) < 1e-12 and rel(H(J2), Jref) < 1e-12, (bx, by, bz, th)
    t = fsi.fsi_mesh_autotune(mesh, 2, fsi.FSI_DF64, reps=2)
    assert len(t["candidates"]) == 10
    _, _, R2, J2 = run(fsi, mesh, "df64", U, A, f, x)
    assert rel(H(R2), Rref) < 1e-12 and rel(H(J2), Jref) < 1e-12
    # 16 x 8 x 4 doubles the per-operator shared memory past the limit
    with pytest.raises(fsi.FsiError):
        fsi.fsi_mesh_set_brick(mesh, 2, fsi.FSI_DF64, 16, 8, 4, 256)


def test_fused_on_a_tetrahedral_mesh_and_aliasing(fsi):
    import torch
    from paper_2601_08266_gb300 import inputs
    X, Tt = inputs.tet_box_mesh(4, seed=2, perturb=0.2)
    mesh = fsi.MeshTet(T(X), T(Tt), rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, has_s=True, device=0)
    U, A, f, x = inputs_for(mesh.n_nodes, 5, "df64")
    R1, J1, R2, J2 = run(fsi, mesh, "df64", U, A, f, x)
    assert torch.equal(R1, R2) and torch.equal(J1, J2)
    Ud = T(U)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_residual_jacobian_apply(mesh, fsi.FSI_DF64, Ud, T(A), None, T(x), Ud,
                                        torch.empty_like(Ud))
    out = torch.empty_like(Ud)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_residual_jacobian_apply(mesh, fsi.FSI_DF64, Ud, T(A), None, T(x), out, out)
