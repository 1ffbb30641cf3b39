"""GPU parity on unstructured meshes of linear tetrahedra: VMS residual and
Jacobian apply, point location (bit-exact elements and barycentric
coordinates), the element -> points table, interpolation and spreading,
against the tetrahedral oracle on the same seeded, shuffled meshes."""
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


@pytest.fixture(scope="module")
def tet(oracle):
    from oracle import tet as t
    return t


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


def PREC(fsi, prec):
    return {"f64": fsi.FSI_F64, "f32": fsi.FSI_F32, "df64": fsi.FSI_DF64}[prec]


def make(fsi, N, seed, perturb=0.25, **phys):
    p = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, has_s=False)
    p.update(phys)
    X, Tt = inputs.tet_box_mesh(N, seed=seed, perturb=perturb)
    mesh = fsi.TetMesh(T(X), T(Tt), **p, device=0)
    return mesh, X, Tt, p


def vms(fsi, mesh, prec, U, A, f, x):
    import torch
    dt = dtype_of(prec)
    Ud, Ad, xd = T(U, dt), T(A, dt), T(x, dt)
    fd = None if f is None else T(f, dt)
    R, Jx = torch.empty_like(Ud), torch.empty_like(Ud)
    fsi.fsi_tet_residual(mesh, PREC(fsi, prec), Ud, Ad, fd, R)
    fsi.fsi_tet_jacobian_apply(mesh, PREC(fsi, prec), Ud, Ad, fd, xd, Jx)
    torch.cuda.synchronize()
    return H(R), H(Jx)


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
@pytest.mark.parametrize("N", [(5, 4, 3), (1, 1, 1), (9, 2, 7)])
def test_tet_vms_parity(fsi, tet, oracle, prec, N):
    """Shuffled, perturbed meshes (elements of both orientations), s field,
    body force, rho != 1, O(1) velocities; the last pass of the launch is
    ragged (element counts not multiples of the 64 elements of a CTA)."""
    mesh, X, Tt, p = make(fsi, N, seed=sum(N), rho=1.3, mu=0.02, dt=0.01, rho_inf=0.3,
                          has_s=True)
    n = mesh.n_nodes
    rng = np.random.default_rng(sum(N) + 1)
    U = rng.uniform(-2, 2, (n, 4))
    A = rng.uniform(-1, 1, (n, 4))
    A[:, 3] = rng.uniform(1.0, 50.0, n)
    f, x = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    U, A, f, x = (cast(prec, a) for a in (U, A, f, x))
    R, Jx = vms(fsi, mesh, prec, U, A, f, x)
    om = tet.TetMesh(cast(prec, X), Tt)
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    eR = rel(R, tet.residual(om, p, U, A, f=f))
    eJ = rel(Jx, tet.jacobian_apply(om, p, U, A, x, c_a, c_v, f=f))
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ
    mesh.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_tet_vms_smooth_fields_16cubed(fsi, tet, oracle, prec):
    """24,576 elements with smooth velocity and pressure, no body force."""
    N = 16
    mesh, X, Tt, p = make(fsi, N, seed=3, perturb=0.2)
    n = mesh.n_nodes
    rng = np.random.default_rng(4)
    k = rng.normal(size=(3, 3))
    U = np.concatenate([np.sin(X @ k), np.cos(X @ k[0])[:, None]], 1)
    A = np.zeros((n, 4))
    A[:, :3] = np.cos(X @ k.T)
    A[:, 3] = 1.0
    x = rng.normal(size=(n, 4))
    U, A, x = (cast(prec, a) for a in (U, A, x))
    R, Jx = vms(fsi, mesh, prec, U, A, None, x)
    om = tet.TetMesh(cast(prec, X), Tt)
    c_a, c_v = oracle.timeint.chain_factors(p["rho_inf"], p["dt"])
    eR = rel(R, tet.residual(om, p, U, A))
    eJ = rel(Jx, tet.jacobian_apply(om, p, U, A, x, c_a, c_v))
    assert eR < TOL[prec], eR
    assert eJ < TOL[prec], eJ
    # deterministic: the same call twice gives the same bits
    R2, J2 = vms(fsi, mesh, prec, U, A, None, x)
    assert np.array_equal(R, R2) and np.array_equal(Jx, J2)
    mesh.close()


def locate_gpu(fsi, mesh, P):
    import torch
    m = P.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    lam = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    nout = fsi.fsi_tet_locate(mesh, T(P), elem, lam, cs, perm)
    torch.cuda.synchronize()
    return elem.cpu().numpy(), H(lam), cs.cpu().numpy(), perm.cpu().numpy(), nout, (elem, lam,
                                                                                   cs, perm)


def test_tet_locate_bit_exact(fsi, tet):
    """Points inside known elements, on faces, edges and nodes, and outside:
    elements, barycentric coordinates and the cell table equal the oracle's
    brute-force search bit for bit (same operations, same order, lowest
    element number among several holders)."""
    mesh, X, Tt, _ = make(fsi, (6, 5, 4), seed=7, perturb=0.25)
    om = tet.TetMesh(X, Tt)
    rng = np.random.default_rng(8)
    k = 1500
    e_true = rng.integers(0, om.n_elems, k)
    lam = rng.dirichlet(np.ones(4), k)
    lam[: k // 4, rng.integers(0, 4)] = 0.0          # on a face
    lam /= lam.sum(axis=1, keepdims=True)
    P = np.einsum("ba,bai->bi", lam, X[Tt[e_true]])
    P = np.concatenate([P, X[rng.integers(0, len(X), 200)], rng.uniform(-0.2, 1.2, (400, 3))])
    e, l3, cs, perm, nout, _ = locate_gpu(fsi, mesh, P)
    eo, lo, nouto = tet.locate(om, P)
    assert nout == nouto and nout > 0
    assert np.array_equal(e, eo)
    assert np.array_equal(l3, lo)
    cso, permo = tet.cell_hash(om, eo)
    assert np.array_equal(cs, cso) and np.array_equal(perm, permo)
    mesh.close()


@pytest.mark.parametrize("prec", ["f64", "f32", "df64"])
def test_tet_interp_spread_parity(fsi, tet, prec):
    import torch
    mesh, X, Tt, _ = make(fsi, (7, 6, 5), seed=9, perturb=0.2)
    om = tet.TetMesh(X, Tt)
    rng = np.random.default_rng(10)
    m = 3000
    P = np.concatenate([0.2 + 0.6 * rng.uniform(size=(m - 100, 3)),
                        rng.uniform(-0.5, 1.5, (100, 3))])
    e, l3, cs, perm, nout, (ed, ld, csd, permd) = locate_gpu(fsi, mesh, P)
    dt = dtype_of(prec)
    U = cast(prec, rng.normal(size=(om.n_nodes, 4)))
    lv = cast(prec, rng.normal(size=(m, 3)))
    w = cast(prec, rng.uniform(0.5, 2.0, m))
    F0 = cast(prec, rng.normal(size=(om.n_nodes, 4)))
    u = torch.empty((m, 3), dtype=dt, device="cuda")
    lw = ld.to(dt)
    fsi.fsi_tet_interp(mesh, PREC(fsi, prec), ed, lw, T(U, dt), u)
    F = T(F0, dt).clone()
    fsi.fsi_tet_spread(mesh, PREC(fsi, prec), ed, lw, csd, permd, T(lv, dt), T(w, dt), F, True)
    F2 = torch.zeros_like(F)
    fsi.fsi_tet_spread(mesh, PREC(fsi, prec), ed, lw, csd, permd, T(lv, dt), None, F2, False)
    torch.cuda.synchronize()
    lo = cast(prec, l3)
    assert rel(H(u), tet.interp(om, e, lo, U)) < TOL[prec]
    Fo = tet.spread(om, e, lo, lv, w=w, F=F0, accumulate=True)
    assert rel(H(F)[:, :3], Fo[:, :3]) < TOL[prec]
    assert np.array_equal(H(F)[:, 3], F0[:, 3])             # pressure slot untouched
    assert rel(H(F2)[:, :3], tet.spread(om, e, lo, lv)[:, :3]) < TOL[prec]
    mesh.close()


def test_tet_empty_and_all_outside(fsi, tet):
    import torch
    mesh, X, Tt, _ = make(fsi, 3, seed=11)
    for P in (np.zeros((0, 3)), np.full((17, 3), 5.0)):
        m = P.shape[0]
        e, l3, cs, perm, nout, (ed, ld, csd, permd) = locate_gpu(fsi, mesh, P)
        assert nout == m and np.all(cs == 0) and np.array_equal(perm, np.arange(m))
        u = torch.ones((m, 3), dtype=torch.float64, device="cuda")
        fsi.fsi_tet_interp(mesh, fsi.FSI_F64, ed, ld, torch.ones((mesh.n_nodes, 4),
                                                                  dtype=torch.float64,
                                                                  device="cuda"), u)
        F = torch.full((mesh.n_nodes, 4), 2.0, dtype=torch.float64, device="cuda")
        fsi.fsi_tet_spread(mesh, fsi.FSI_F64, ed, ld, csd, permd,
                           torch.ones((m, 3), dtype=torch.float64, device="cuda"), None, F, False)
        torch.cuda.synchronize()
        assert np.all(H(u) == 0.0)
        assert np.all(H(F)[:, :3] == 0.0) and np.all(H(F)[:, 3] == 2.0)
    mesh.close()


def test_tet_mesh_rejects_bad_input(fsi):
    import torch
    X, Tt = inputs.tet_box_mesh(2, seed=0)
    bad = Tt.copy()
    bad[3, 1] = len(X) + 5
    with pytest.raises(fsi.FsiError):
        fsi.TetMesh(T(X), T(bad), device=0)
    with pytest.raises(ValueError):
        fsi.TetMesh(T(X[:, :2].copy()), T(Tt), device=0)
