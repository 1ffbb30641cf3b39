"""The Krylov solver's multi-dot (Sec. 2.4: the Gram-Schmidt dot products
stay FP64): FP32 basis vectors, products formed exactly and summed on the
FP32 pipe with compensation, against the exact sums of the same FP32 values
(math.fsum of their FP64 products, which are exact)."""
import math

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


@pytest.mark.parametrize("length,nvec", [(4, 1), (4 * 1000, 3), (4 * 250_003, 11)])
def test_multi_dot_is_fp64_grade(fsi, length, nvec):
    import torch
    from paper_2601_08266_gb300 import _binding as B
    rng = np.random.default_rng(length + nvec)
    # wide dynamic range and heavy cancellation: the sums are far below the
    # sums of magnitudes
    scale = np.exp(rng.uniform(-8, 8, size=length))
    w = (rng.normal(size=length) * scale).astype(np.float32)
    V = (rng.normal(size=(nvec, length)) * scale[None, :]).astype(np.float32)
    V[0] -= (V[0] @ w.astype(np.float64)) / (w.astype(np.float64) @ w) * w  # near-orthogonal
    V = V.astype(np.float32)
    Vd, wd = torch.as_tensor(V, device="cuda"), torch.as_tensor(w, device="cuda")
    out = torch.empty(nvec, dtype=torch.float64, device="cuda")
    B.fsi_multi_dot(B.FSI_F32, Vd, wd, out)
    got = out.cpu().numpy()
    out2 = torch.empty_like(out)
    B.fsi_multi_dot(B.FSI_F32, Vd, wd, out2)
    assert np.array_equal(got, out2.cpu().numpy())   # fixed reduction order
    for k in range(nvec):
        prods = V[k].astype(np.float64) * w.astype(np.float64)   # exact in FP64
        exact = math.fsum(prods)
        mag = math.fsum(np.abs(prods))
        assert abs(got[k] - exact) <= 2.0 ** -40 * mag, (k, got[k], exact, mag)
    # FP64 vectors: the plain FP64 sums
    out64 = torch.empty_like(out)
    B.fsi_multi_dot(B.FSI_F64, Vd.double(), wd.double(), out64)
    ref = V.astype(np.float64) @ w.astype(np.float64)
    mags = np.abs(V.astype(np.float64)) @ np.abs(w.astype(np.float64))
    assert np.all(np.abs(out64.cpu().numpy() - ref) <= 1e-13 * mags)
