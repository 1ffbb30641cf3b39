"""Local parity measures for comparing a CUDA result with the oracle's.

One relative norm over a whole output can hide a wrong subset: the
continuity row of a nodal field is much smaller than its momentum rows, the
nodes on one face of the box are a few percent of all nodes, and a few
thousand wrong entries barely move the 2-norm of a million.  So every
operator parity test measures each part on its own:

  * component groups: for a nodal [n][4] array the momentum rows 0..2 and the
    continuity (or pressure) row 3; any other array is one group;
  * regions, where the structured grid is known: the nodes on the faces of
    the box and the interior nodes;
  * for every (group, region) part S, the norm-wise error
    ||gpu_S - ref_S||_2 / ||ref_S||_2 and the largest entry error
    max|gpu_S - ref_S| / max|ref_S|.

rel_local returns the worst of these numbers, so a test keeps its tolerance
(1e-12 for FP64 and double-float, 1e-5 for FP32) and now holds it on every
part.  A part whose reference is identically zero is measured against the
whole group's reference instead (its entries must then be tiny, not exact).
"""
from __future__ import annotations

import numpy as np


def boundary_mask(N):
    """True for the nodes on a face of the (Nx, Ny, Nz)-element box, in the
    lexicographic node order (x fastest)."""
    Nx, Ny, Nz = (N, N, N) if np.isscalar(N) else N
    i = np.arange(Nx + 1)
    j = np.arange(Ny + 1)
    k = np.arange(Nz + 1)
    bi = (i == 0) | (i == Nx)
    bj = (j == 0) | (j == Ny)
    bk = (k == 0) | (k == Nz)
    return (bk[:, None, None] | bj[None, :, None] | bi[None, None, :]).ravel()


def local_errors(got, ref, grid=None):
    """{(group, region, measure): error} for the parts described above."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    if got.shape != ref.shape:
        raise AssertionError(f"shape {got.shape} != {ref.shape}")
    if ref.ndim == 1:
        got, ref = got[:, None], ref[:, None]
    elif ref.ndim > 2:
        got, ref = got.reshape(len(got), -1), ref.reshape(len(ref), -1)
    if ref.shape[1] == 4:
        groups = {"momentum": slice(0, 3), "continuity": slice(3, 4)}
    else:
        groups = {"all": slice(0, ref.shape[1])}
    regions = {"all": np.ones(len(ref), dtype=bool)}
    if grid is not None:
        b = boundary_mask(grid)
        if len(b) == len(ref):
            regions = {"boundary": b, "interior": ~b}
    out = {}
    for gname, cols in groups.items():
        rg = ref[:, cols]
        g2 = np.linalg.norm(rg)
        gi = np.abs(rg).max() if rg.size else 0.0
        for rname, rows in regions.items():
            if not rows.any():
                continue
            r = ref[rows][:, cols]
            d = got[rows][:, cols] - r
            n2 = np.linalg.norm(r) or g2 or 1.0
            ni = (np.abs(r).max() if r.size else 0.0) or gi or 1.0
            out[(gname, rname, "l2")] = float(np.linalg.norm(d) / n2)
            out[(gname, rname, "max")] = float(np.abs(d).max() / ni) if d.size else 0.0
    return out


def rel_local(got, ref, grid=None):
    """The worst local error of got against ref (0 for empty arrays)."""
    errs = local_errors(got, ref, grid)
    return max(errs.values()) if errs else 0.0


def worst(got, ref, grid=None):
    """(error, part) of the worst part, for messages."""
    errs = local_errors(got, ref, grid)
    if not errs:
        return 0.0, None
    k = max(errs, key=errs.get)
    return errs[k], k
