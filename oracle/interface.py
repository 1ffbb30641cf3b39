"""Interface scaling field s of Sec. 2.1, plain.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.1 multiplies the bracket of tau_M by a scaling s that is much larger
than 1 in an O(h) neighbourhood of the fluid-solid interface and 1 elsewhere,
defined at the fluid nodes and interpolated with the pressure's (Q1) basis, so
that the transition is smooth over one element.  Reading (the paper fixes no
band width): the neighbourhood is the set of cells that contain a solid point,
dilated by `layers` cells in every direction (Chebyshev distance in cell
indices, clipped at the grid); every node of a band cell gets s = s_band, every
other node s = 1.

Pins (tests/test_oracle_interface.py): one point gives its cell's 8 nodes
(layers = 0) or the (2 layers + 2)^3 nodes around it; clipping at the grid
boundary; the band of a point set is the union of the bands of its points; the
field only takes the values 1 and s_band.
"""
from __future__ import annotations

import numpy as np

from . import core


def occupied_cells(grid: core.Grid, elem):
    """Boolean [Nz, Ny, Nx]: cells that contain at least one located point."""
    occ = np.zeros(grid.n_elems, dtype=bool)
    e = np.asarray(elem)
    occ[e[e >= 0]] = True
    return occ.reshape(grid.N[2], grid.N[1], grid.N[0])


def band_cells(grid: core.Grid, elem, layers: int):
    """Occupied cells dilated by `layers` cells (Chebyshev distance), by loops."""
    occ = occupied_cells(grid, elem)
    Nx, Ny, Nz = grid.N
    band = np.zeros_like(occ)
    for k, j, i in zip(*np.nonzero(occ)):
        band[max(0, k - layers):min(Nz, k + layers + 1),
             max(0, j - layers):min(Ny, j + layers + 1),
             max(0, i - layers):min(Nx, i + layers + 1)] = True
    return band


def scaling_field(grid: core.Grid, elem, s_band: float, layers: int = 0):
    """s [n] at the nodes: s_band on every node of a band cell, 1 elsewhere."""
    band = band_cells(grid, elem, layers)
    Nx, Ny, Nz = grid.N
    on = np.zeros((Nz + 1, Ny + 1, Nx + 1), dtype=bool)
    for dk in (0, 1):
        for dj in (0, 1):
            for di in (0, 1):
                on[dk:dk + Nz, dj:dj + Ny, di:di + Nx] |= band
    return np.where(on.ravel(), float(s_band), 1.0)
