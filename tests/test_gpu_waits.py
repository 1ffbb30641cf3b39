"""Failure detection without a GPU fault: the bounded wait that the
tensor-core kernels use gives up on a planted mbarrier that nothing
completes, the kernel reports it through its error flag, and the context
keeps working."""
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


def test_bounded_wait_runs_out_and_the_context_stays_usable(fsi, oracle):
    import torch
    timed_out, seconds = fsi.fsi_wait_selftest(0)
    assert timed_out, "the planted wait did not run out"
    assert 0.0 < seconds < 30.0, seconds
    # the same context runs library kernels afterwards, with correct results
    mesh = fsi.Mesh(4, device=0)
    rng = np.random.default_rng(0)
    U, A = rng.normal(size=(mesh.n_nodes, 4)), rng.normal(size=(mesh.n_nodes, 4))
    A[:, 3] = 1.0
    R = torch.empty((mesh.n_nodes, 4), dtype=torch.float64, device="cuda")
    fsi.fsi_residual(mesh, fsi.FSI_F64, torch.as_tensor(U, device="cuda"),
                     torch.as_tensor(A, device="cuda"), None, R)
    torch.cuda.synchronize()
    p = dict(rho=1.0, mu=0.01, dt=1e-3, rho_inf=0.5, has_s=False)
    ref = oracle.core.residual(oracle.core.Grid(4), p, U, A)
    assert np.linalg.norm(R.cpu().numpy() - ref) <= 1e-12 * np.linalg.norm(ref)
    mesh.close()
