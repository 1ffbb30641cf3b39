"""GPU parity of point location and the cell -> points table, bit for bit
against the oracle, on the cases the uniform-grid kernels branch on:

- spacings that are powers of two (location by integer work on the bits of
  the coordinates) with zero and non-zero origins, and points on the faces,
  just inside and outside them (one ulp), at signed zeros, subnormals,
  infinities and NaN;
- grids of more than 1024 scan tiles (2048 cells each: the tile sums are
  scanned by one CTA first) and of fewer;
- cells of one point, 2 to 128 points (placed by the rank pass) and more
  (the CTA-sorted dense list), the tail of outside points among them (the
  in-place variant of the table, without point scratch, is covered through
  fsi_locate_noalloc and the tetrahedral mesh);
- repeated calls on one mesh with changing point sets (the per-cell counters
  and the scan scratch are left at zero by every call).
"""
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


def run_locate(fsi, mesh, X):
    import torch
    m = X.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(mesh.n_elems + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    Xd = torch.as_tensor(np.ascontiguousarray(X), device="cuda")
    nout = fsi.fsi_locate(mesh, Xd, elem, xi, cs, perm)
    torch.cuda.synchronize()
    return elem.cpu().numpy(), xi.cpu().numpy(), cs.cpu().numpy(), perm.cpu().numpy(), nout


def check(fsi, oracle, mesh, grid, X):
    e, xi, cs, perm, nout = run_locate(fsi, mesh, X)
    eo, xio, nouto = oracle.core.locate(grid, X)
    cso, permo = oracle.core.cell_hash(grid, eo)
    assert nout == nouto
    assert np.array_equal(e, eo)
    # bit patterns, so that -0.0 against 0.0 and NaN payloads would show
    assert np.array_equal(xi.view(np.int64), xio.view(np.int64))
    assert np.array_equal(cs, cso)
    assert np.array_equal(perm, permo)
    return nout


def edge_points(N, h, x0, rng):
    """Points on and one ulp either side of every grid plane of each axis,
    special values, and random points, per axis combined with random
    in-range coordinates of the other axes."""
    cols = []
    for k in range(3):
        planes = x0[k] + h[k] * np.arange(N[k] + 1)
        vals = np.concatenate([planes, np.nextafter(planes, -np.inf),
                               np.nextafter(planes, np.inf),
                               [0.0, -0.0, 5e-324, -5e-324, 2.2e-308, np.inf, -np.inf, np.nan,
                                x0[k] + h[k] * N[k] * 1e-17]])
        cols.append(vals)
    pts = []
    for k in range(3):
        v = cols[k]
        P = np.empty((v.size, 3))
        for a in range(3):
            P[:, a] = (x0[a] + h[a] * N[a] * rng.uniform(0, 1, v.size)) if a != k else v
        pts.append(P)
    lo, hi = np.array(x0), np.array(x0) + np.array(h) * np.array(N)
    pts.append(lo + (hi - lo) * rng.uniform(-0.05, 1.05, (4000, 3)))
    return np.concatenate(pts)


@pytest.mark.parametrize("x0", [(0.0, 0.0, 0.0), (0.25, -0.5, 0.0), (-0.0, 3.0, -2.0)])
def test_locate_power_of_two_spacings(fsi, oracle, x0):
    rng = np.random.default_rng(31)
    N, h = (16, 8, 32), (2.0 ** -4, 2.0 ** -3, 1.0)
    mesh = fsi.Mesh(N, x0=x0, h=h, device=0)
    grid = oracle.core.Grid(N, x0=x0, h=h)
    X = edge_points(N, h, x0, rng)
    nout = check(fsi, oracle, mesh, grid, X)
    assert 0 < nout < X.shape[0]


def test_locate_spacing_above_one(fsi, oracle):
    """h = 2 (1/h < 1) takes the division path; results still exact."""
    rng = np.random.default_rng(32)
    N, h, x0 = (5, 6, 7), (2.0, 0.5, 4.0), (1.0, 0.0, -3.0)
    mesh = fsi.Mesh(N, x0=x0, h=h, device=0)
    grid = oracle.core.Grid(N, x0=x0, h=h)
    check(fsi, oracle, mesh, grid, edge_points(N, h, x0, rng))


def clustered_points(N, rng):
    """Cells with 1, 2..32, 33..128 and > 128 points, in segments (32
    consecutive cells) of up to 32, 33..128 and more points, plus scattered
    points and outside points, in shuffled order."""
    Nx, Ny, Nz = N
    h = 1.0 / np.array(N, dtype=np.float64)

    def in_cell(i, j, k, n):
        c = np.array([i, j, k], dtype=np.float64)
        return (c + rng.uniform(0.01, 0.99, (n, 3))) * h

    parts = [
        in_cell(3, 4, 5, 200),        # a dense cell (CTA sort)
        in_cell(4, 4, 5, 129),        # just over the rank pass's limit
        in_cell(9, 2, 2, 128),        # exactly 128
        in_cell(10, 2, 2, 40),
        in_cell(20, 7, 3, 33),
    ]
    # neighbouring cells of a few points each
    for i in range(0, 24, 3):
        parts.append(in_cell(i, 11, 6, 9))
    for i in range(0, 32, 4):
        parts.append(in_cell(i, 13, 1, 3))
    parts.append(rng.uniform(0, 1, (20000, 3)))
    parts.append(rng.uniform(1.01, 2.0, (300, 3)))   # outside: the tail cell
    X = np.concatenate(parts)
    return X[rng.permutation(X.shape[0])]


def test_cell_table_segments_and_dense_cells(fsi, oracle):
    rng = np.random.default_rng(33)
    N = (48, 40, 36)
    mesh = fsi.Mesh(N, device=0)
    grid = oracle.core.Grid(N)
    X = clustered_points(N, rng)
    check(fsi, oracle, mesh, grid, X)
    # outside points beyond a warp's limit: a dense tail cell
    Xo = np.concatenate([X, rng.uniform(2.0, 3.0, (500, 3))])
    check(fsi, oracle, mesh, grid, Xo[rng.permutation(Xo.shape[0])])


def test_cell_table_many_tiles_and_repeated_calls(fsi, oracle):
    """128 x 128 x 200 cells = 1600 scan tiles; the same mesh then serves
    changing point sets (more, fewer, none, all outside) and must give the
    oracle's table each time."""
    rng = np.random.default_rng(34)
    N = (128, 128, 200)
    mesh = fsi.Mesh(N, device=0)
    grid = oracle.core.Grid(N)
    L = inputs.leaflet_points(300_000, seed=35)
    sets = [L, L[:1000], np.zeros((0, 3)), np.full((77, 3), -1.0),
            np.concatenate([L[::3], rng.uniform(-0.1, 1.1, (50_000, 3))]), L]
    for X in sets:
        check(fsi, oracle, mesh, grid, X)


def test_cell_table_fewer_tiles(fsi, oracle):
    """A grid of 1 scan tile and one of exactly 1024 tiles (128^3)."""
    rng = np.random.default_rng(36)
    for N in ((3, 4, 5), (128, 128, 128)):
        mesh = fsi.Mesh(N, device=0)
        grid = oracle.core.Grid(N)
        X = rng.uniform(-0.02, 1.02, (60_000, 3))
        check(fsi, oracle, mesh, grid, X)
        check(fsi, oracle, mesh, grid, X[:5000])

