"""GPU parity of the Schur-complement preconditioner's pressure multigrid
(pmg.cu) against the assembled oracle (oracle/precond.py): hierarchy, operator,
transfers, Chebyshev smoother and the whole V-cycle; and its effect inside the
Newton step."""
import numpy as np
import pytest

import parity

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def fsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08266_gb300 as pkg
    return pkg


def T(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda").to(dtype).contiguous()


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


def dtype_of(prec):
    import torch
    return torch.float64 if prec == "f64" else torch.float32


def cast(prec, a):
    return a.astype(np.float32).astype(np.float64) if prec == "f32" else a


GRIDS = [((8, 8, 8), None), ((14, 14, 14), None), ((6, 5, 7), (0.2, 0.1, 0.1)),
         ((16, 8, 12), (0.05, 0.1, 0.0625)), ((32, 32, 32), None)]


FACES = [(0,) * 6, (0, 1, 0, 0, 1, 0), (1,) * 6]


def setup(fsi, N, h, faces=(0,) * 6):
    from oracle import precond as pc
    hh = tuple(1.0 / v for v in N) if h is None else h
    mesh = fsi.Mesh(N, h=h, device=0)
    fsi.fsi_pressure_set_faces(mesh, faces)
    mg = pc.MultigridOracle(N, hh, faces=faces)
    return mesh, mg


@pytest.mark.parametrize("N,h", GRIDS[:4])
def test_hierarchy_matches_oracle(fsi, N, h):
    mesh, mg = setup(fsi, N, h)
    assert fsi.fsi_pressure_levels(mesh) == [L.N for L in mg.levels]


@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("N,h", GRIDS[:4])
def test_operator_and_transfers_match_oracle(fsi, prec, N, h, faces):
    import torch
    mesh, mg = setup(fsi, N, h, faces)
    dt = dtype_of(prec)
    rng = np.random.default_rng(7)
    for l, L in enumerate(mg.levels):
        x = cast(prec, rng.normal(size=L.n))
        y = torch.empty(L.n, dtype=dt, device="cuda")
        fsi.fsi_pressure_apply(mesh, l, T(x, dt), y)
        torch.cuda.synchronize()
        assert rel(H(y), mg.A[l] @ x) < TOL[prec], (l, prec)
        if l + 1 < len(mg.levels):
            nc = mg.levels[l + 1].n
            b = torch.empty(nc, dtype=dt, device="cuda")
            fsi.fsi_pressure_restrict(mesh, l, T(x, dt), b)
            xc = cast(prec, rng.normal(size=nc))
            base = cast(prec, rng.normal(size=L.n))
            xf = T(base, dt)
            fsi.fsi_pressure_prolong_add(mesh, l, T(xc, dt), xf)
            torch.cuda.synchronize()
            ref_b = mg.P[l].T @ x
            ref_b[mg.dirn[l + 1]] = 0.0
            assert rel(H(b), ref_b) < TOL[prec]
            assert rel(H(xf), base + mg.P[l] @ xc) < TOL[prec]


@pytest.mark.parametrize("faces", FACES[:2])
@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_smoother_matches_oracle(fsi, prec, faces):
    import torch
    mesh, mg = setup(fsi, (8, 8, 8), None, faces)
    dt = dtype_of(prec)
    rng = np.random.default_rng(3)
    n = mg.levels[0].n
    b = cast(prec, rng.normal(size=n))
    x0 = cast(prec, rng.normal(size=n))
    for deg in (1, 2, 5):
        x = torch.empty(n, dtype=dt, device="cuda")
        fsi.fsi_pressure_smooth(mesh, 0, deg, T(b, dt), x, from_zero=True)
        ref = mg.smooth(0, b, np.zeros(n), degree=deg)
        xs = T(x0, dt)
        fsi.fsi_pressure_smooth(mesh, 0, deg, T(b, dt), xs, from_zero=False)
        ref2 = mg.smooth(0, b, x0, degree=deg)
        torch.cuda.synchronize()
        assert rel(H(x), ref) < TOL[prec], deg
        assert rel(H(xs), ref2) < TOL[prec], deg


@pytest.mark.parametrize("faces", FACES)
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("N,h", GRIDS)
def test_vcycle_matches_oracle(fsi, prec, N, h, faces):
    import torch
    mesh, mg = setup(fsi, N, h, faces)
    dt = dtype_of(prec)
    n = mg.levels[0].n
    b = cast(prec, np.random.default_rng(11).normal(size=n))
    x = torch.empty(n, dtype=dt, device="cuda")
    fsi.fsi_pressure_vcycle(mesh, T(b, dt), x)
    torch.cuda.synchronize()
    ref = mg.vcycle(b)
    assert rel(H(x), ref) < (TOL[prec] if prec == "f64" else 2e-5), (N, prec)


def test_vcycle_rejects_aliasing_and_bad_levels(fsi):
    import torch
    mesh, _ = setup(fsi, (8, 8, 8), None)
    v = torch.zeros(729, dtype=torch.float64, device="cuda")
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_vcycle(mesh, v, v)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_apply(mesh, 5, v, v.clone())
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_restrict(mesh, 1, v, v.clone())   # level 1 is the coarsest


def test_schur_preconditioner_cuts_krylov_iterations(fsi, oracle):
    """Same Newton step, both preconditioners: the same converged solution,
    and the Schur preconditioner needs far fewer Krylov iterations.  The
    Newton tolerance is 1e-10 so that the two iterates, each stopped just
    below it, lie within 1e-5 of one another."""
    import torch
    from paper_2601_08266_gb300 import inputs
    N, dt = 24, 1e-3
    n = (N + 1) ** 3
    rng = np.random.default_rng(2)
    ax = np.arange(N + 1) / N
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    X, Y, Z = X.ravel(), Y.ravel(), Z.ravel()
    wall = (Y < 1e-12) | (Y > 1 - 1e-12) | (Z < 1e-12) | (Z > 1 - 1e-12)
    inflow = (X < 1e-12) & ~wall
    mask = np.zeros((n, 4), dtype=np.uint8)
    mask[wall | inflow, :3] = 1
    prof = 16 * Y * (1 - Y) * Z * (1 - Z)
    Vn = np.zeros((n, 4))
    Vn[:, 0] = prof
    Vn[:, :3] += 0.05 * rng.normal(size=(n, 3))
    Vn[mask[:, 0].astype(bool), :3] = 0
    Vn[inflow, 0] = prof[inflow]
    An = np.zeros((n, 4))
    yD = np.zeros((n, 4))
    m = 20000
    Xp = inputs.leaflet_points(m, seed=5)
    res = {}
    for pc in (fsi.PRECOND_BLOCK_JACOBI, fsi.PRECOND_SCHUR):
        for mixed in (False, True):
            mesh = fsi.Mesh(N, rho=1.0, mu=1e-3, dt=dt, rho_inf=0.5, device=0)
            e = torch.empty(m, dtype=torch.int32, device="cuda")
            xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
            cs = torch.empty(N ** 3 + 1, dtype=torch.int32, device="cuda")
            pm = torch.empty(m, dtype=torch.int32, device="cuda")
            fsi.fsi_locate(mesh, T(Xp, torch.float64), e, xi, cs, pm)
            y = torch.zeros((n, 4), dtype=torch.float64, device="cuda")
            st = fsi.StepState(y, T(Vn, torch.float64), T(An, torch.float64),
                               mask=T(mask, torch.uint8), yD=T(yD, torch.float64), elem=e, xi=xi,
                               cell_start=cs, perm=pm,
                               w=torch.full((m,), 0.024 / m, dtype=torch.float64, device="cuda"),
                               drho_s=0.5)
            code, rep = fsi.fsi_newton_step(mesh, st, mixed=mixed, restart=50, max_newton=10,
                                            max_krylov=4000, newton_rtol=1e-10, krylov_rtol=1e-3,
                                            precond=pc)
            assert code == 0 and rep["converged"], rep
            res[(pc, mixed)] = (rep["krylov_iters"], H(y))
    for mixed in (False, True):
        kj, yj = res[(fsi.PRECOND_BLOCK_JACOBI, mixed)]
        ks, ys = res[(fsi.PRECOND_SCHUR, mixed)]
        print(f"\nN={N} mixed={mixed}: Krylov iterations block-Jacobi {kj}, Schur {ks}")
        assert ks * 2 < kj, (kj, ks)
        assert rel(ys, yj) < 1e-5
