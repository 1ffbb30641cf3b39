"""The algebraic-multigrid pressure block on a structured grid
(fsi_pressure_use_amg; Sec. 2.4's Schur approximation with the operator
assembled on a mapped grid): the level-0 operator against the oracle's Q1
assembly at the mapped coordinates, with and without eliminated nodes; on a
uniform grid it equals the geometric multigrid's operator; the V-cycle as a
symmetric positive definite preconditioner; the switch and its invalidation
by new coordinates."""
import numpy as np
import pytest

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


def coords(N, h, amp, seed):
    ax = [h[d] * np.arange(N[d] + 1) for d in range(3)]
    Z, Y, X = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    P = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    i, j, k = (P / np.asarray(h)).round().astype(int).T
    inn = (i > 0) & (i < N[0]) & (j > 0) & (j < N[1]) & (k > 0) & (k < N[2])
    rng = np.random.default_rng(seed)
    P[inn] += amp * rng.uniform(-1, 1, (inn.sum(), 3)) * np.asarray(h)[None, :]
    return P, ~inn


def make(fsi, N, amp, seed, eliminate):
    from oracle import precond
    h = tuple(1.0 / N[d] for d in range(3))
    X, bnd = coords(N, h, amp, seed)
    mesh = fsi.Mesh(N, h=h, rho=1.0, mu=0.05, dt=0.01, rho_inf=0.5, device=0)
    if amp > 0:
        mesh.set_coordinates(T(X))
    fsi.fsi_pressure_use_amg(mesh, True)
    el = None
    if eliminate:
        el = bnd & (X[:, 2] > 0.5)
        fsi.fsi_pressure_set_eliminated(mesh, T(el.astype(np.uint8)))
    return mesh, precond.mapped_pressure_operator(N, X, eliminated=el), el


def apply(fsi, mesh, level, x):
    import torch
    y = torch.empty_like(x)
    fsi.fsi_pressure_apply(mesh, level, x, y)
    return y


@pytest.mark.parametrize("eliminate", [False, True])
@pytest.mark.parametrize("N,amp", [((6, 5, 7), 0.0), ((6, 5, 7), 0.3), ((13, 9, 11), 0.25)])
def test_level0_operator_matches_the_oracle(fsi, N, amp, eliminate):
    import torch
    mesh, A, el = make(fsi, N, amp, seed=3, eliminate=eliminate)
    x = np.random.default_rng(1).normal(size=A.shape[0])
    y_ref = A @ x
    y64 = H(apply(fsi, mesh, 0, T(x)))
    assert np.abs(y64 - y_ref).max() <= 1e-12 * np.abs(y_ref).max()
    y32 = H(apply(fsi, mesh, 0, T(x, torch.float32)))
    assert np.abs(y32 - y_ref).max() <= 1e-5 * np.abs(y_ref).max()
    if amp == 0.0 and not eliminate:
        # the geometric multigrid's level-0 operator on the same uniform grid
        fsi.fsi_pressure_use_amg(mesh, False)
        yg = H(apply(fsi, mesh, 0, T(x)))
        assert np.abs(yg - y64).max() <= 1e-12 * np.abs(y_ref).max()


@pytest.mark.parametrize("eliminate", [False, True])
def test_vcycle_is_an_spd_preconditioner(fsi, eliminate):
    import torch
    import scipy.sparse.linalg as sla
    mesh, A, _ = make(fsi, (20, 18, 22), 0.3, seed=6, eliminate=eliminate)
    n = A.shape[0]
    sizes = fsi.fsi_pressure_level_sizes(mesh)
    assert sizes[0] == n and len(sizes) >= 2 and sizes[-1] <= 600
    rng = np.random.default_rng(7)
    b1, b2 = T(rng.normal(size=n)), T(rng.normal(size=n))
    v1, v2 = torch.empty_like(b1), torch.empty_like(b2)
    fsi.fsi_pressure_vcycle(mesh, b1, v1)
    fsi.fsi_pressure_vcycle(mesh, b2, v2)
    a, b = float(v1 @ b2), float(b1 @ v2)
    assert abs(a - b) <= 1e-10 * (abs(a) + abs(b))
    assert float(v1 @ b1) > 0 and float(v2 @ b2) > 0
    assert pcg(fsi, mesh, A, rng) <= 25


def pcg(fsi, mesh, A, rng, max_its=100):
    """Conjugate gradients on the level-0 operator preconditioned by one
    V-cycle; the iterations to a 1e-8 relative residual (the solution is
    checked against a direct solve)."""
    import torch
    import scipy.sparse.linalg as sla
    n = A.shape[0]
    b = T(rng.normal(size=n))
    x = torch.zeros_like(b)
    r = b.clone()
    z = torch.empty_like(b)
    fsi.fsi_pressure_vcycle(mesh, r, z)
    p, rz, its = z.clone(), float(r @ z), 0
    while float(r.norm()) > 1e-8 * float(b.norm()) and its < max_its:
        Ap = apply(fsi, mesh, 0, p)
        alpha = rz / float(p @ Ap)
        x += alpha * p
        r -= alpha * Ap
        fsi.fsi_pressure_vcycle(mesh, r, z)
        rz_new = float(r @ z)
        p = z + (rz_new / rz) * p
        rz = rz_new
        its += 1
    xr = sla.spsolve(A.tocsc(), H(b))
    assert np.abs(H(x) - xr).max() <= 1e-6 * np.abs(xr).max()
    return its


@pytest.mark.parametrize("N,amp", [((32, 8, 16), 0.0), ((16, 16, 4), 0.2), ((20, 18, 22), 0.4)])
def test_vcycle_on_anisotropic_and_strongly_mapped_grids(fsi, N, amp, capsys):
    """Cells of aspect ratio 4 (h_x : h_y = 1 : 4, and h_z = 4 h_x with a
    mapping) and strongly distorted cells (nodes moved by up to 0.4 h: the
    smallest Gauss-point Jacobian is 6 % of the undistorted one; at 0.45 h this
    seed inverts some): the Q1 couplings change size and sign there, yet the
    aggregation must still coarsen (at least two levels, a small coarsest
    level) and the V-cycle keep preconditioned CG short."""
    mesh, A, _ = make(fsi, N, amp, seed=11, eliminate=False)
    sizes = fsi.fsi_pressure_level_sizes(mesh)
    its = pcg(fsi, mesh, A, np.random.default_rng(12))
    with capsys.disabled():
        print(f"\nAMG N={N} amp={amp}: levels {sizes}, PCG iterations {its}")
    assert sizes[0] == A.shape[0] and len(sizes) >= 2 and sizes[-1] <= 600, sizes
    assert sizes[1] <= sizes[0] // 4, sizes
    assert its <= 40, its


def test_switch_and_new_coordinates(fsi):
    from oracle import precond
    N = (5, 6, 4)
    mesh, A, _ = make(fsi, N, 0.2, seed=8, eliminate=False)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_levels(mesh)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_set_faces(mesh, (1, 0, 0, 0, 0, 0))
    x = T(np.random.default_rng(2).normal(size=A.shape[0]))
    assert np.abs(H(apply(fsi, mesh, 0, x)) - A @ H(x)).max() <= 1e-12 * abs(A).max()
    # new coordinates: the hierarchy is rebuilt from them
    h = tuple(1.0 / N[d] for d in range(3))
    X2, _ = coords(N, h, 0.35, seed=9)
    mesh.set_coordinates(T(X2))
    A2 = precond.mapped_pressure_operator(N, X2)
    assert np.abs(H(apply(fsi, mesh, 0, x)) - A2 @ H(x)).max() <= 1e-12 * abs(A2).max()
    # back to the geometric multigrid: its calls work again, set_eliminated refuses
    fsi.fsi_pressure_use_amg(mesh, False)
    assert fsi.fsi_pressure_levels(mesh)
    with pytest.raises(fsi.FsiError):
        fsi.fsi_pressure_set_eliminated(mesh, None)
