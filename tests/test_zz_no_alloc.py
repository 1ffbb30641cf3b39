"""Point location for callers that cannot allocate device memory.

Some callers of this library must not call cudaMalloc: code running inside a
host application whose memory manager owns all device memory, and loops that
cannot afford the implicit device-wide synchronisation of an allocation.  For
them fsi_locate_noalloc works without a mesh handle and keeps its scratch in a
static device array.  These tests call it through the C ABI twice in a row (a
large grid, then a small anisotropic one, so the second call starts from the
first call's leftover scratch) and check that its outputs are bit-identical to
those of fsi_locate, and that grids beyond the array's limit are refused.
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


def _locate_both(fsi, N, h, x0, X):
    import torch
    m = X.shape[0]
    E = N[0] * N[1] * N[2]
    Xd = torch.as_tensor(X, device="cuda").contiguous()
    outs = []
    for which in ("mesh", "noalloc"):
        elem = torch.full((m,), 7, dtype=torch.int32, device="cuda")
        xi = torch.full((m, 3), 3.0, dtype=torch.float64, device="cuda")
        cs = torch.full((E + 1,), -5, dtype=torch.int32, device="cuda")
        perm = torch.full((m,), -5, dtype=torch.int32, device="cuda")
        if which == "mesh":
            mesh = fsi.Mesh(N, x0=x0, h=h, device=0)
            nout = fsi.fsi_locate(mesh, Xd, elem, xi, cs, perm)
        else:
            nout = fsi.fsi_locate_noalloc(N, x0, h, Xd, elem, xi, cs, perm, device=0)
        torch.cuda.synchronize()
        outs.append((nout, elem.cpu().numpy(), xi.cpu().numpy(), cs.cpu().numpy(),
                     perm.cpu().numpy()))
    return outs


def test_noalloc_locate_matches_fsi_locate_on_two_calls(fsi):
    cases = [((64, 64, 64), (1 / 64,) * 3, (0.0, 0.0, 0.0),
              np.concatenate([inputs.leaflet_points(200_000, seed=31),
                              inputs.edge_points(64, seed=2, m_random=500)])),
             ((13, 9, 21), (0.08, 0.1, 0.05), (-0.1, 0.05, 0.0),
              inputs.edge_points((13, 9, 21), seed=3, m_random=4000) * np.array([1.1, 0.95, 1.1]))]
    for N, h, x0, X in cases:
        ref, got = _locate_both(fsi, N, h, x0, X)
        assert got[0] == ref[0]
        for a, b in zip(got[1:], ref[1:]):
            assert np.array_equal(a, b)


def test_noalloc_locate_refuses_grids_beyond_its_scratch(fsi):
    import torch
    X = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    elem = torch.empty(4, dtype=torch.int32, device="cuda")
    xi = torch.empty((4, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(fsi.FsiError) as e:
        fsi.fsi_locate_noalloc((200, 200, 200), (0, 0, 0), (0.005,) * 3, X, elem, xi)
    assert e.value.status == 1 and "maximum" in str(e.value)
