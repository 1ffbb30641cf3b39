"""GPU parity of the immersed hyperelastic solid (solid.cu, Sec. 2.2) against
oracle/solid.py: nodal residual, tangent, generalized-alpha staging, and the
coupled reduced system with the body inside the Newton step."""
import numpy as np
import pytest

import parity

pytestmark = pytest.mark.gpu

MAT = dict(rho_s=1.6, rho_f=1.0, mu=40.0, lam=150.0)


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
    return t.to(dtype).contiguous() if dtype is not None else t


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


def body_mesh(n=(4, 3, 2), lo=(0.3, 0.3, 0.35), hi=(0.7, 0.6, 0.55), amp=0.01, seed=0):
    from oracle import solid as so
    m = so.box_mesh(n, lo, hi)
    m.X = m.X + amp * np.random.default_rng(seed).uniform(-1, 1, m.X.shape)
    return m


def make_solid(fsi, mesh, m):
    import torch
    return fsi.Solid(mesh, T(m.X, torch.float64), T(m.conn.astype(np.int32), torch.int32),
                     MAT["rho_s"], MAT["mu"], MAT["lam"])


def test_solid_residual_and_tangent_match_oracle(fsi):
    import torch
    from oracle import solid as so
    mesh = fsi.Mesh(8, rho=MAT["rho_f"], mu=0.05, dt=0.01, rho_inf=0.5, device=0)
    m = body_mesh()
    b = make_solid(fsi, mesh, m)
    rng = np.random.default_rng(1)
    u_af, u_n = 0.03 * rng.normal(size=(m.ns, 3)), 0.02 * rng.normal(size=(m.ns, 3))
    v_af, a_am = rng.normal(size=(m.ns, 3)), rng.normal(size=(m.ns, 3))
    g = (0.0, -9.81, 0.5)
    R = torch.empty((m.ns, 3), dtype=torch.float64, device="cuda")
    fsi.fsi_solid_residual(b, T(u_af), T(v_af), T(a_am), T(u_n), g, R)
    torch.cuda.synchronize()
    ref = so.residual(m, u_af, v_af, a_am, u_n, MAT, 0.05, g)
    assert rel(H(R), ref) < 1e-12
    x = rng.normal(size=(m.ns, 3))
    ca, cu, cv = so.chain(0.01)
    Jref = so.tangent_apply(m, u_af, u_n, x, MAT, 0.05, ca, cu, cv)
    for prec, dt, tol in ((fsi.FSI_F64, torch.float64, 1e-12), (fsi.FSI_F32, torch.float32, 1e-5)):
        xx = x.astype(np.float32).astype(np.float64) if dt == torch.float32 else x
        uu = u_af.astype(np.float32).astype(np.float64) if dt == torch.float32 else u_af
        Jx = torch.empty((m.ns, 3), dtype=dt, device="cuda")
        fsi.fsi_solid_tangent_apply(b, prec, T(uu, dt), T(u_n), T(xx, dt), Jx)
        torch.cuda.synchronize()
        assert rel(H(Jx), so.tangent_apply(m, uu, u_n, xx, MAT, 0.05, ca, cu, cv)) < tol
    assert rel(so.tangent_apply(m, u_af, u_n, x, MAT, 0.05, ca, cu, cv), Jref) == 0.0
    b.close()


def test_solid_stage_and_advance_match_oracle(fsi):
    import torch
    from oracle import solid as so
    mesh = fsi.Mesh(4, dt=0.013, rho_inf=0.5, device=0)
    m = body_mesh(n=(2, 2, 1))
    b = make_solid(fsi, mesh, m)
    rng = np.random.default_rng(2)
    u, v, a, a1 = (rng.normal(size=(m.ns, 3)) for _ in range(4))
    outs = [torch.empty((m.ns, 3), dtype=torch.float64, device="cuda") for _ in range(3)]
    fsi.fsi_solid_stage(b, T(u), T(v), T(a), T(a1), *outs)
    ud, vd, ad = T(u), T(v), T(a)
    fsi.fsi_solid_advance(b, ud, vd, ad, T(a1))
    torch.cuda.synchronize()
    u_af, v_af, a_am, u_next, v_next = so.kinematics(u, v, a, a1, 0.013)
    for got, ref in zip(outs + [ud, vd, ad], [u_af, v_af, a_am, u_next, v_next, a1]):
        assert rel(H(got), ref) < 1e-14
    b.close()


def coupled_setup(fsi, oracle, N=8, seed=3, dt=0.05):
    import torch
    from oracle import newton, solid as so
    grid = oracle.core.Grid(N)
    n = grid.n_nodes
    rng = np.random.default_rng(seed)
    m = body_mesh(n=(3, 2, 2), seed=seed)
    us, vs, as_ = (0.01 * rng.normal(size=(m.ns, 3)), 0.1 * rng.normal(size=(m.ns, 3)),
                   rng.normal(size=(m.ns, 3)))
    phys = dict(rho=1.0, mu=0.05, dt=dt, rho_inf=0.5)
    Vn, An = 0.3 * rng.normal(size=(n, 4)), 0.3 * rng.normal(size=(n, 4))
    Xn = grid.node_coords()
    bnd = np.any((Xn < 1e-12) | (Xn > 1 - 1e-12), axis=1)
    mask = np.zeros((n, 4), dtype=bool)
    mask[bnd, :3] = True
    mask[0, 3] = True
    yD = np.zeros((n, 4))
    g = (0.0, 0.0, -1.0)
    body = dict(mesh=m, u=us, v=vs, a=as_, mat=MAT, g=g)
    P = newton.Problem(grid, phys, Vn, An, mask=mask, yD=yD, body=body)
    y = rng.normal(size=(n, 4))
    y[mask] = 0.0
    mesh = fsi.Mesh(N, rho=1.0, mu=0.05, dt=dt, rho_inf=0.5, device=0)
    b = make_solid(fsi, mesh, m)
    xs = torch.empty((m.ns, 3), dtype=torch.float64, device="cuda")
    fsi.fsi_solid_positions(b, T(us), xs)
    e = torch.empty(m.ns, dtype=torch.int32, device="cuda")
    xi = torch.empty((m.ns, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    pm = torch.empty(m.ns, dtype=torch.int32, device="cuda")
    fsi.fsi_locate(mesh, xs, e, xi, cs, pm)
    dev = dict(y=T(y), Vn=T(Vn), An=T(An), mask=T(mask.astype(np.uint8)), yD=T(yD),
               us=T(us), vs=T(vs), as_=T(as_))
    st = fsi.StepState(dev["y"], dev["Vn"], dev["An"], mask=dev["mask"], yD=dev["yD"], elem=e,
                       xi=xi, cell_start=cs, perm=pm, g_s=g, body=b, us=dev["us"], vs=dev["vs"],
                       as_=dev["as_"])
    return mesh, b, st, dev, P, y


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_coupled_residual_with_the_body_matches_oracle(fsi, oracle, prec):
    import torch
    mesh, b, st, dev, P, y = coupled_setup(fsi, oracle)
    R = torch.empty_like(dev["y"])
    fsi.fsi_coupled_residual(mesh, st, R, prec=fsi.FSI_F64 if prec == "f64" else fsi.FSI_DF64)
    torch.cuda.synchronize()
    assert rel(H(R), P.residual(y)) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coupled_jacobian_with_the_body_matches_oracle(fsi, oracle, prec):
    import torch
    mesh, b, st, dev, P, y = coupled_setup(fsi, oracle)
    x = np.random.default_rng(9).normal(size=y.shape)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    R = torch.empty_like(dev["y"])
    fsi.fsi_coupled_residual(mesh, st, R)     # sets the linearisation point
    Jx = torch.empty(y.shape, dtype=dt, device="cuda")
    fsi.fsi_coupled_jacobian_apply(mesh, fsi.FSI_F64 if prec == "f64" else fsi.FSI_F32, st,
                                   T(x, dt), Jx)
    torch.cuda.synchronize()
    ref = (P.jacobian(y) @ x.ravel()).reshape(y.shape)
    assert rel(H(Jx), ref) < (1e-12 if prec == "f64" else 1e-5)


@pytest.mark.parametrize("mixed", [False, True])
def test_newton_step_with_the_body_matches_direct_newton(fsi, oracle, mixed):
    from oracle import newton
    mesh, b, st, dev, P, y0 = coupled_setup(fsi, oracle, seed=5)
    code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=12,
                                    max_krylov=3000, newton_rtol=1e-8, krylov_rtol=1e-3)
    assert code == 0 and rep["converged"] == 1, rep
    y_gpu = H(dev["y"])
    assert np.linalg.norm(P.residual(y_gpu)) <= 1.01e-8 * rep["r_ref"]
    y_ref, _ = newton.newton(P, y0, rtol=1e-13)
    assert rel_norm(y_gpu, y_ref) < 5e-5, rep
