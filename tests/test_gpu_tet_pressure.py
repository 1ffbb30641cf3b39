"""The pressure block of the Schur-complement preconditioner on a tetrahedral
mesh (Sec. 2.4): the level-0 operator K + kappa M against the oracle's P1
assembly, with and without eliminated nodes; the algebraic-multigrid levels
(restriction the transpose of prolongation, Galerkin coarse operators); the
V-cycle as a symmetric positive definite preconditioner that makes conjugate
gradients converge in few iterations; and the Newton step with the Schur
preconditioner landing on the oracle's direct-solve solution."""
import numpy as np
import pytest

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


def make(fsi, N, seed, eliminate):
    from oracle import tet
    X, Tt = inputs.tet_box_mesh(N, seed=seed, perturb=0.2)
    mesh = fsi.MeshTet(T(X), T(Tt), rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, device=0)
    el = None
    if eliminate:
        el = np.any(X > 1 - 1e-12, axis=1) | (np.any(X < 1e-12, axis=1) & (X[:, 2] > 0.5))
        fsi.fsi_pressure_set_eliminated(mesh, T(el.astype(np.uint8)))
    L = np.ptp(X, axis=0).max()
    kappa = (np.pi / (2.0 * L)) ** 2
    A = tet.pressure_operator(tet.TetMesh(X, Tt), kappa, eliminated=el)
    return mesh, A, el


def apply(fsi, mesh, level, x):
    import torch
    y = torch.empty_like(x)
    fsi.fsi_pressure_apply(mesh, level, x, y)
    return y


@pytest.mark.parametrize("eliminate", [False, True])
@pytest.mark.parametrize("N", [5, (14, 11, 9)])
def test_level0_operator_matches_the_oracle(fsi, N, eliminate):
    import torch
    mesh, A, el = make(fsi, N, seed=3, eliminate=eliminate)
    n = A.shape[0]
    x = np.random.default_rng(1).normal(size=n)
    y_ref = A @ x
    y64 = H(apply(fsi, mesh, 0, T(x)))
    assert np.abs(y64 - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    y32 = H(apply(fsi, mesh, 0, T(x, torch.float32)))
    assert np.abs(y32 - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    if eliminate:
        d = A.diagonal()
        assert np.abs(y64[el] - d[el] * x[el]).max() <= 1e-12 * np.abs(y_ref).max()


@pytest.mark.parametrize("eliminate", [False, True])
def test_levels_restriction_and_galerkin_operators(fsi, eliminate):
    import torch
    mesh, A, _ = make(fsi, 16, seed=4, eliminate=eliminate)
    sizes = fsi.fsi_pressure_level_sizes(mesh)
    assert sizes[0] == A.shape[0] and len(sizes) >= 2
    assert all(b < a for a, b in zip(sizes, sizes[1:]))
    assert sizes[-1] <= 600
    rng = np.random.default_rng(5)
    for l in range(len(sizes) - 1):
        nf, nc = sizes[l], sizes[l + 1]
        r, xc = T(rng.normal(size=nf)), T(rng.normal(size=nc))
        Rr = torch.empty(nc, dtype=torch.float64, device="cuda")
        fsi.fsi_pressure_restrict(mesh, l, r, Rr)
        Pxc = torch.zeros(nf, dtype=torch.float64, device="cuda")
        fsi.fsi_pressure_prolong_add(mesh, l, xc, Pxc)
        # <R r, xc> = <r, P xc>
        a, b = float(Rr @ xc), float(r @ Pxc)
        assert abs(a - b) <= 1e-12 * max(abs(a), 1.0) * nf
        # A_{l+1} xc = R A_l P xc
        lhs = H(apply(fsi, mesh, l + 1, xc))
        APx = apply(fsi, mesh, l, Pxc)
        rhs = torch.empty(nc, dtype=torch.float64, device="cuda")
        fsi.fsi_pressure_restrict(mesh, l, APx, rhs)
        rhs = H(rhs)
        assert np.abs(lhs - rhs).max() <= 1e-11 * np.abs(rhs).max()


def pcg(fsi, mesh, b, tol, maxit=200):
    import torch
    x = torch.zeros_like(b)
    r = b.clone()
    z = torch.empty_like(b)
    fsi.fsi_pressure_vcycle(mesh, r, z)
    p = z.clone()
    rz = float(r @ z)
    nb = float(b.norm())
    for k in range(1, maxit + 1):
        Ap = apply(fsi, mesh, 0, p)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        if float(r.norm()) <= tol * nb:
            return x, k
        fsi.fsi_pressure_vcycle(mesh, r, z)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x, maxit + 1


@pytest.mark.parametrize("eliminate", [False, True])
def test_vcycle_is_an_spd_preconditioner(fsi, eliminate):
    import torch
    mesh, A, _ = make(fsi, 24, seed=6, eliminate=eliminate)
    n = A.shape[0]
    rng = np.random.default_rng(7)
    b1, b2 = T(rng.normal(size=n)), T(rng.normal(size=n))
    v1, v2 = torch.empty_like(b1), torch.empty_like(b2)
    fsi.fsi_pressure_vcycle(mesh, b1, v1)
    fsi.fsi_pressure_vcycle(mesh, b2, v2)
    a, b = float(v1 @ b2), float(b1 @ v2)
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))
    assert float(v1 @ b1) > 0 and float(v2 @ b2) > 0
    # deterministic
    v1b = torch.empty_like(b1)
    fsi.fsi_pressure_vcycle(mesh, b1, v1b)
    assert torch.equal(v1, v1b)
    b = T(rng.normal(size=n))
    x, its = pcg(fsi, mesh, b, 1e-8)
    assert its <= 25, its
    import scipy.sparse.linalg as sla
    xr = sla.spsolve(A.tocsc(), H(b))
    assert np.abs(H(x) - xr).max() <= 1e-6 * np.abs(xr).max()
    # FP32 V-cycle agrees with the FP64 one to FP32 rounding
    v32 = torch.empty(n, dtype=torch.float32, device="cuda")
    fsi.fsi_pressure_vcycle(mesh, b1.float(), v32)
    assert np.abs(H(v32) - H(v1)).max() <= 1e-4 * np.abs(H(v1)).max()


def test_smoother_reduces_the_error(fsi):
    import torch
    mesh, A, _ = make(fsi, 12, seed=8, eliminate=True)
    n = A.shape[0]
    xs = np.random.default_rng(9).normal(size=n)
    b = T(A @ xs)
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    Ad = A.toarray()
    e0 = xs @ Ad @ xs
    fsi.fsi_pressure_smooth(mesh, 0, 8, b, x, True)
    e = xs - H(x)
    e1 = e @ Ad @ e
    fsi.fsi_pressure_smooth(mesh, 0, 8, b, x, False)
    e = xs - H(x)
    e2 = e @ Ad @ e
    assert e1 < e0 and e2 < e1


def test_structured_only_calls_refuse_a_tetrahedral_mesh(fsi):
    mesh, _, _ = make(fsi, 4, seed=1, eliminate=False)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_levels(mesh)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_set_faces(mesh, [1, 0, 0, 0, 0, 0])


def test_set_eliminated_refuses_a_structured_grid(fsi):
    import torch
    mesh = fsi.Mesh(4, h=0.25, rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, device=0)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_set_eliminated(mesh, torch.zeros(125, dtype=torch.uint8, device="cuda"))


def test_every_node_eliminated_and_back(fsi):
    """All nodes eliminated: the operator is its diagonal, no aggregate forms,
    the hierarchy has one level and the V-cycle still returns a bounded
    approximation of D^-1 b; clearing the set rebuilds the full hierarchy."""
    import torch
    mesh, A, _ = make(fsi, 12, seed=10, eliminate=False)
    n = A.shape[0]
    full = fsi.fsi_pressure_level_sizes(mesh)
    assert len(full) >= 2
    fsi.fsi_pressure_set_eliminated(mesh, torch.ones(n, dtype=torch.uint8, device="cuda"))
    assert fsi.fsi_pressure_level_sizes(mesh) == [n]
    b = T(np.random.default_rng(11).normal(size=n))
    x = torch.empty_like(b)
    fsi.fsi_pressure_vcycle(mesh, b, x)
    d = A.diagonal()
    xr = H(b) / d
    assert np.all(np.isfinite(H(x)))
    assert np.linalg.norm(H(x) - xr) <= 0.2 * np.linalg.norm(xr)
    fsi.fsi_pressure_set_eliminated(mesh, None)
    assert fsi.fsi_pressure_level_sizes(mesh) == full
