"""Point location for callers that cannot allocate device memory.

Some callers of this library must not call cudaMalloc: code running inside a
host application whose memory manager owns all device memory, and loops that
cannot afford the implicit device-wide synchronisation of an allocation.  For
them fsi_locate_noalloc works without a mesh handle and keeps its scratch in a
static device array.  These tests call it through the C ABI twice in a row (a
large grid, then a small anisotropic one, so the second call starts from the
first call's leftover scratch) and check that its outputs are bit-identical to
those of fsi_locate, with and without the cell table, for an empty point set
and in strict mode with points outside the grid; that a call leaves the
device's free memory unchanged; and that grids beyond the array's limit,
including extents whose product overflows 32 bits, are refused before any
launch.
"""
import numpy as np
import pytest

from paper_2601_08266_gb300 import inputs
from paper_2601_08266_gb300._binding import FSI_ERR_OUTSIDE

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fsi():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2601_08266_gb300 as pkg
    return pkg


def _run(fsi, which, N, h, x0, Xd, table, strict):
    """One call of fsi_locate (on a fresh mesh) or fsi_locate_noalloc; returns
    (status, n_outside, elem, xi, cell_start, perm) with the outputs that were
    requested, pre-filled with junk so that unwritten entries show."""
    import torch
    m = Xd.shape[0]
    E = N[0] * N[1] * N[2]
    elem = torch.full((m,), 7, dtype=torch.int32, device="cuda")
    xi = torch.full((m, 3), 3.0, dtype=torch.float64, device="cuda")
    cs = torch.full((E + 1,), -5, dtype=torch.int32, device="cuda") if table else None
    perm = torch.full((m,), -5, dtype=torch.int32, device="cuda") if table else None
    status, nout = 0, None
    try:
        if which == "mesh":
            mesh = fsi.Mesh(N, x0=x0, h=h, device=0)
            nout = fsi.fsi_locate(mesh, Xd, elem, xi, cs, perm, strict=strict)
        else:
            nout = fsi.fsi_locate_noalloc(N, x0, h, Xd, elem, xi, cs, perm, strict=strict,
                                          device=0)
    except fsi.FsiError as e:
        status = e.status
    torch.cuda.synchronize()
    host = lambda t: None if t is None else t.cpu().numpy()
    return status, nout, host(elem), host(xi), host(cs), host(perm)


def _same(fsi, N, h, x0, X, table=True, strict=False):
    import torch
    Xd = torch.as_tensor(X, device="cuda").reshape(-1, 3).contiguous()
    ref = _run(fsi, "mesh", N, h, x0, Xd, table, strict)
    got = _run(fsi, "noalloc", N, h, x0, Xd, table, strict)
    assert got[0] == ref[0] and got[1] == ref[1]
    for a, b in zip(got[2:], ref[2:]):
        assert (a is None and b is None) or np.array_equal(a, b)
    return got


CASES = [((64, 64, 64), (1 / 64,) * 3, (0.0, 0.0, 0.0),
          lambda: np.concatenate([inputs.leaflet_points(200_000, seed=31),
                                  inputs.edge_points(64, seed=2, m_random=500)])),
         ((13, 9, 21), (0.08, 0.1, 0.05), (-0.1, 0.05, 0.0),
          lambda: inputs.edge_points((13, 9, 21), seed=3, m_random=4000)
          * np.array([1.1, 0.95, 1.1]))]


def test_noalloc_locate_matches_fsi_locate_on_two_calls(fsi):
    for N, h, x0, make in CASES:
        _same(fsi, N, h, x0, make())


@pytest.mark.parametrize("table", [True, False])
def test_noalloc_locate_paths(fsi, table):
    """Without the cell table, an empty point set, and strict mode with
    points outside the grid (FSI_ERR_OUTSIDE after all outputs are written):
    the same statuses and outputs as fsi_locate."""
    N, h, x0, make = CASES[1]
    X = make()
    got = _same(fsi, N, h, x0, X, table=table)
    assert got[1] > 0
    inside = X[got[2] >= 0]
    _same(fsi, N, h, x0, np.zeros((0, 3)), table=table)
    got = _same(fsi, N, h, x0, X, table=table, strict=True)
    assert got[0] == FSI_ERR_OUTSIDE
    got = _same(fsi, N, h, x0, inside, table=table, strict=True)
    assert got[0] == 0 and got[1] == 0


def test_noalloc_locate_allocates_nothing(fsi):
    """After a first call on the device (which may load the library's module
    and with it the static array), further calls leave the device's free
    memory unchanged: the call allocates nothing."""
    import torch
    N, h, x0, make = CASES[0]
    Xd = torch.as_tensor(make(), device="cuda").contiguous()
    m = Xd.shape[0]
    elem = torch.empty(m, dtype=torch.int32, device="cuda")
    xi = torch.empty((m, 3), dtype=torch.float64, device="cuda")
    cs = torch.empty(N[0] * N[1] * N[2] + 1, dtype=torch.int32, device="cuda")
    perm = torch.empty(m, dtype=torch.int32, device="cuda")
    fsi.fsi_locate_noalloc(N, x0, h, Xd, elem, xi, cs, perm, device=0)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info(0)
    for _ in range(2):
        fsi.fsi_locate_noalloc(N, x0, h, Xd, elem, xi, cs, perm, device=0)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info(0)
    assert free1 == free0


@pytest.mark.parametrize("N", [(200, 200, 200), (1 << 21, 1 << 21, 1 << 22),
                               (1 << 16, 1 << 16, 1), (4_000_001, 1, 1)])
def test_noalloc_locate_refuses_grids_beyond_its_scratch(fsi, N):
    import torch
    X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    elem = torch.empty(4, dtype=torch.int32, device="cuda")
    xi = torch.empty((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_locate_noalloc(N, (0, 0, 0), (0.005,) * 3, X, elem, xi)
    assert e.value.status == 1 and "maximum" in str(e.value)
