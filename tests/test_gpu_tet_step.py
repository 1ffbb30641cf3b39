"""The implicit step on a tetrahedral mesh through the step's own entry points
(an fsi_mesh backed by a tetrahedral mesh): the operators equal the
tetrahedral ones, the coupled residual, Jacobian and probed diagonal blocks
match the oracle's coupled problem, and the Newton step (plain FP64 and mixed,
block-Jacobi or the Schur-complement preconditioner) lands on the oracle's
direct-solve solution."""
import numpy as np
import pytest

import parity

from paper_2601_08266_gb300 import inputs

pytestmark = pytest.mark.gpu


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


def setup(fsi, oracle, N=4, m=200, seed=0, dt=0.01, mu=0.05):
    import torch
    from oracle import newton, tet
    X, Tt = inputs.tet_box_mesh(N, seed=seed, perturb=0.2)
    om = tet.TetMesh(X, Tt)
    n = om.n_nodes
    rng = np.random.default_rng(seed + 1)
    phys = dict(rho=1.0, mu=mu, dt=dt, rho_inf=0.5, has_s=True)
    Vn, An = 0.5 * rng.normal(size=(n, 4)), 0.5 * rng.normal(size=(n, 4))
    s = rng.uniform(1.0, 3.0, n)
    f = rng.normal(size=(n, 4))
    P = inputs.ball_points(m, seed=seed + 2, radius=0.3)
    elem, lam, nout = tet.locate(om, P)
    assert nout == 0
    w = rng.uniform(0.5, 1.5, m)
    bnd = np.any((X < 1e-12) | (X > 1 - 1e-12), axis=1)
    mask = np.zeros((n, 4), dtype=bool)
    mask[bnd, :3] = True
    mask[0, 3] = True
    yD = np.zeros((n, 4))
    yD[bnd, :3] = 0.3 * rng.normal(size=(int(bnd.sum()), 3))
    solid = dict(drho=0.7, k=2.0, g=(0.0, 0.0, -9.81))
    prob = newton.Problem(om, phys, Vn, An, f=f, s=s, mask=mask, yD=yD, points=(elem, lam, w),
                          solid=solid)
    y = rng.normal(size=(n, 4))
    y[mask] = yD[mask]
    mesh = fsi.MeshTet(T(X), T(Tt), rho=1.0, mu=mu, dt=dt, rho_inf=0.5, has_s=True, device=0)
    e_d = torch.empty(m, dtype=torch.int32, device="cuda")
    l_d = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs_d = torch.empty(om.n_elems + 1, dtype=torch.int32, device="cuda")
    pm_d = torch.empty(m, dtype=torch.int32, device="cuda")
    assert fsi.fsi_locate(mesh, T(P), e_d, l_d, cs_d, pm_d) == 0
    assert np.array_equal(e_d.cpu().numpy(), elem)
    dev = dict(y=T(y), Vn=T(Vn), An=T(An), s=T(s), f=T(f), mask=T(mask.astype(np.uint8)),
               yD=T(yD), w=T(w))
    st = fsi.StepState(dev["y"], dev["Vn"], dev["An"], s=dev["s"], f=dev["f"], mask=dev["mask"],
                       yD=dev["yD"], elem=e_d, xi=l_d, cell_start=cs_d, perm=pm_d, w=dev["w"],
                       drho_s=0.7, k_s=2.0, g_s=(0.0, 0.0, -9.81))
    return mesh, st, dev, prob, y, om


def test_step_entry_points_equal_the_tetrahedral_ones(fsi, oracle):
    import torch
    X, Tt = inputs.tet_box_mesh((5, 4, 3), seed=3, perturb=0.2)
    mesh = fsi.MeshTet(T(X), T(Tt), has_s=True, device=0)
    tm = fsi.TetMesh(T(X), T(Tt), has_s=True, device=0)
    n = len(X)
    rng = np.random.default_rng(4)
    Uh, Ah, xh = (rng.normal(size=(n, 4)) for _ in range(3))
    Ah[:, 3] = rng.uniform(1.0, 3.0, n)          # the band s is positive
    U, A, x = T(Uh), T(Ah), T(xh)
    out = []
    for handle, res, jac in ((mesh, fsi.fsi_residual, fsi.fsi_jacobian_apply),
                             (tm, fsi.fsi_tet_residual, fsi.fsi_tet_jacobian_apply)):
        R, J = torch.empty_like(U), torch.empty_like(U)
        res(handle, fsi.FSI_DF64, U, A, None, R)
        jac(handle, fsi.FSI_DF64, U, A, None, x, J)
        out.append((R.clone(), J.clone()))
    torch.cuda.synchronize()
    assert torch.isfinite(out[0][0]).all() and torch.isfinite(out[0][1]).all()
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    # structured-only features refuse the handle
    with pytest.raises(fsi.FsiError):
        fsi.fsi_mesh_set_coordinates(mesh, T(X))


@pytest.mark.parametrize("prec", ["f64", "df64"])
def test_coupled_residual_parity(fsi, oracle, prec):
    import torch
    mesh, st, dev, prob, y, _ = setup(fsi, oracle)
    R = torch.empty_like(dev["y"])
    fsi.fsi_coupled_residual(mesh, st, R, prec=fsi.FSI_F64 if prec == "f64" else fsi.FSI_DF64)
    torch.cuda.synchronize()
    assert rel(H(R), prob.residual(y)) < 1e-12


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_coupled_jacobian_and_diagonal_blocks(fsi, oracle, prec):
    import torch
    mesh, st, dev, prob, y, om = setup(fsi, oracle, dt=0.05)
    n = om.n_nodes
    x = np.random.default_rng(9).normal(size=y.shape)
    dt = torch.float64 if prec == "f64" else torch.float32
    if prec == "f32":
        x = x.astype(np.float32).astype(np.float64)
    Jx = torch.empty(y.shape, dtype=dt, device="cuda")
    P = fsi.FSI_F64 if prec == "f64" else fsi.FSI_F32
    fsi.fsi_coupled_jacobian_apply(mesh, P, st, T(x, dt), Jx)
    B = torch.empty((n, 4, 4), dtype=dt, device="cuda")
    fsi.fsi_block_diagonal(mesh, P, st, B)
    torch.cuda.synchronize()
    J = prob.jacobian(y).tocsr()
    tol = 1e-12 if prec == "f64" else 1e-5
    assert rel(H(Jx), (J @ x.ravel()).reshape(y.shape)) < tol
    ref = np.zeros((n, 4, 4))
    for a in range(n):
        ref[a] = J[4 * a:4 * a + 4, 4 * a:4 * a + 4].toarray()
    assert rel(H(B), ref) < tol


@pytest.mark.parametrize("mixed", [False, True])
def test_newton_step_on_a_tetrahedral_mesh(fsi, oracle, mixed):
    from oracle import newton
    mesh, st, dev, prob, y0, _ = setup(fsi, oracle, seed=5)
    code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=12,
                                    max_krylov=4000, newton_rtol=1e-8, krylov_rtol=1e-3,
                                    precond=fsi.PRECOND_BLOCK_JACOBI)
    assert code == 0 and rep["converged"] == 1, rep
    y_gpu = H(dev["y"])
    assert np.linalg.norm(prob.residual(y_gpu)) <= 1.01e-8 * rep["r_ref"]
    y_ref, _ = newton.newton(prob, y0, rtol=1e-13)
    assert rel_norm(y_gpu, y_ref) < 5e-5, rep


@pytest.mark.parametrize("mixed", [False, True])
@pytest.mark.parametrize("N", [4, 8])
def test_newton_step_with_the_schur_preconditioner(fsi, oracle, mixed, N):
    """The Schur-complement preconditioner with the algebraic multigrid for
    the pressure (one level at N = 4, two or more at N = 8): the step lands on
    the oracle's direct-solve solution in fewer Krylov iterations than with
    block-Jacobi."""
    from oracle import newton
    its = {}
    for precond in (fsi.PRECOND_BLOCK_JACOBI, fsi.PRECOND_SCHUR):
        mesh, st, dev, prob, y0, _ = setup(fsi, oracle, N=N, seed=7)
        code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=12,
                                        max_krylov=4000, newton_rtol=1e-8, krylov_rtol=1e-3,
                                        precond=precond)
        assert code == 0 and rep["converged"] == 1, (precond, rep)
        its[precond] = rep["krylov_iters"]
        y_gpu = H(dev["y"])
        assert np.linalg.norm(prob.residual(y_gpu)) <= 1.01e-8 * rep["r_ref"]
    y_ref, _ = newton.newton(prob, y0, rtol=1e-13)
    assert rel_norm(y_gpu, y_ref) < 5e-5
    if N == 8:
        assert len(fsi.fsi_pressure_level_sizes(mesh)) >= 2
    assert its[fsi.PRECOND_SCHUR] < its[fsi.PRECOND_BLOCK_JACOBI], its
