"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module only draws random numbers and lays out geometry; it holds none of
the method's arithmetic (no shape functions, no residual, no time
integration).  Everything is numpy float64 on the host.

Workload shapes follow the paper's problems: a uniform background hex grid on
the unit cube, immersed thin leaflet-like solids sampled as point clouds (the
paper's valve leaflets are 0.015-0.0212 thick), and random multipliers.

Recipes (every array is drawn from ``numpy.random.default_rng(seed)``):

* ``uniform_state``   -- nodal unknown y ~ U[-1, 1] i.i.d., history zero.
* ``fourier_field``   -- per component a sum of separable sinusoids with
  wavenumbers 1..8 per axis and random phases/amplitudes, normalised to
  max |v| = 1, plus N(0, 0.01^2) noise.
* ``ball_points``     -- points uniform in a ball.
* ``leaflet_points``  -- three cylindrical-sector shells about the x axis
  through (0.5, 0.5): radius 0.29..0.31, x in [0.1, 0.9], arc 0.5 at radius
  0.3 (95.5 deg), centred 120 deg apart, uniform in volume.
* ``multipliers``     -- lambda ~ N(0, 1) per component.
"""
from __future__ import annotations

import math

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def n_nodes(N) -> int:
    if np.isscalar(N):
        N = (N, N, N)
    return (N[0] + 1) * (N[1] + 1) * (N[2] + 1)


def uniform_state(N, seed: int, lo: float = -1.0, hi: float = 1.0):
    """y[n,4] ~ U[lo,hi] and zero history (Vn, An) -- the one-step workload."""
    g = rng(seed)
    n = n_nodes(N)
    y = g.uniform(lo, hi, size=(n, 4))
    Vn = np.zeros((n, 4))
    An = np.zeros((n, 4))
    return y, Vn, An


def uniform_nodal(N, seed: int, ncomp: int = 4, lo: float = -1.0, hi: float = 1.0):
    g = rng(seed)
    return g.uniform(lo, hi, size=(n_nodes(N), ncomp))


def fourier_field(N, seed: int, modes: int = 8, noise: float = 0.01, ncomp: int = 4):
    """Smooth random field on the nodes of an N^3 unit-cube grid, [n, ncomp]."""
    if np.isscalar(N):
        N = (N, N, N)
    g = rng(seed)
    ax = [np.arange(N[k] + 1) / N[k] for k in range(3)]
    k = np.arange(1, modes + 1)
    out = np.empty((n_nodes(N), ncomp))
    for c in range(ncomp):
        S = []
        for d in range(3):
            ph = g.uniform(0.0, 2.0 * math.pi, size=modes)
            S.append(np.sin(2.0 * math.pi * np.outer(ax[d], k) + ph[None, :]))
        amp = g.normal(size=(modes, modes, modes)) / (1.0 + k[:, None, None] ** 2
                                                     + k[None, :, None] ** 2
                                                     + k[None, None, :] ** 2)
        # field[z, y, x] = sum_{kz,ky,kx} amp[kx,ky,kz] Sx[x,kx] Sy[y,ky] Sz[z,kz]
        f = np.einsum("abc,xa,yb,zc->zyx", amp, S[0], S[1], S[2], optimize=True)
        f /= np.abs(f).max()
        f += g.normal(scale=noise, size=f.shape)
        out[:, c] = f.ravel()
    return out


def ball_points(m: int, seed: int, center=(0.5, 0.5, 0.5), radius: float = 0.3):
    g = rng(seed)
    d = g.normal(size=(m, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    r = radius * g.uniform(0.0, 1.0, size=m) ** (1.0 / 3.0)
    return np.asarray(center)[None, :] + r[:, None] * d


def leaflet_points(m: int, seed: int, theta0: float | None = None, radius: float = 0.3,
                   thickness: float = 0.02, length: float = 0.8, arc: float = 0.5,
                   axis_center=(0.5, 0.5)):
    """m points uniform in the volume of three thin cylindrical-sector shells."""
    g = rng(seed)
    if theta0 is None:
        theta0 = g.uniform(0.0, 2.0 * math.pi)
    which = g.integers(0, 3, size=m)
    half = 0.5 * arc / radius
    r0, r1 = radius - 0.5 * thickness, radius + 0.5 * thickness
    r = np.sqrt(g.uniform(r0 * r0, r1 * r1, size=m))
    th = theta0 + which * (2.0 * math.pi / 3.0) + g.uniform(-half, half, size=m)
    x = g.uniform(0.5 - 0.5 * length, 0.5 + 0.5 * length, size=m)
    y = axis_center[0] + r * np.cos(th)
    z = axis_center[1] + r * np.sin(th)
    return np.stack([x, y, z], axis=1)


def multipliers(m: int, seed: int):
    return rng(seed).normal(size=(m, 3))


def edge_points(N, seed: int, m_random: int = 64):
    """Points on nodes, faces, edges, corners, the far boundary and outside."""
    if np.isscalar(N):
        N = (N, N, N)
    g = rng(seed)
    pts = []
    for i in (0, N[0] // 2, N[0]):
        for j in (0, N[1]):
            for k in (0, N[2] // 3, N[2]):
                pts.append((i / N[0], j / N[1], k / N[2]))
    pts += [(0.5, 0.5, 1.0), (1.0, 1.0, 1.0), (0.0, 0.0, 0.0), (1.0, 0.25, 0.5)]
    pts += [(-1e-9, 0.5, 0.5), (0.5, 1.0 + 1e-9, 0.5), (0.5, 0.5, 2.0), (-3.0, -3.0, -3.0)]
    pts += [(float("nan"), 0.5, 0.5)]
    R = g.uniform(-0.1, 1.1, size=(m_random, 3))
    return np.concatenate([np.asarray(pts, dtype=np.float64), R], axis=0)


def leaflet_hex_mesh(n_r: int, n_theta: int, n_x: int, seed: int, theta0: float | None = None,
                     radius: float = 0.3, thickness: float = 0.02, x_range=(0.1, 0.9),
                     arc: float = 0.5):
    """The three leaflet shells of leaflet_points as a trilinear hexahedral solid
    mesh: per leaflet n_r x n_theta x n_x elements over r in [radius -
    thickness/2, radius + thickness/2], its arc and x_range.  Returns (X [ns, 3],
    conn [es, 8] int32) with corners a = ar + 2 atheta + 4 ax ordered so that
    every element has a positive Jacobian."""
    g = rng(seed)
    if theta0 is None:
        theta0 = g.uniform(0.0, 2.0 * math.pi)
    half = 0.5 * arc / radius
    r = np.linspace(radius - 0.5 * thickness, radius + 0.5 * thickness, n_r + 1)
    xs = np.linspace(x_range[0], x_range[1], n_x + 1)
    X_all, conn_all = [], []
    base = 0
    for which in range(3):
        c = theta0 + which * (2.0 * math.pi / 3.0)
        th = np.linspace(c - half, c + half, n_theta + 1)
        # node (ir, it, ix) -> index ir + (n_r+1) (it + (n_theta+1) ix)
        XX, TT, RR = np.meshgrid(xs, th, r, indexing="ij")
        pts = np.stack([XX.ravel(), 0.5 + RR.ravel() * np.cos(TT.ravel()),
                        0.5 + RR.ravel() * np.sin(TT.ravel())], axis=1)
        X_all.append(pts)
        nr1, nt1 = n_r + 1, n_theta + 1
        ir, it, ix = np.meshgrid(np.arange(n_r), np.arange(n_theta), np.arange(n_x), indexing="ij")
        n0 = ir + nr1 * (it + nt1 * ix)
        corners = [n0 + (a & 1) + nr1 * ((a >> 1) & 1) + nr1 * nt1 * ((a >> 2) & 1)
                   for a in range(8)]
        conn_all.append(np.stack([cc.ravel() for cc in corners], axis=1) + base)
        base += pts.shape[0]
    return np.concatenate(X_all), np.concatenate(conn_all).astype(np.int32)


def tet_box_mesh(N, seed: int, perturb: float = 0.0, shuffle: bool = True, lo=(0.0, 0.0, 0.0),
                 hi=(1.0, 1.0, 1.0)):
    """Unstructured tetrahedral mesh of a box: the N^3 (or Nx x Ny x Nz) grid
    split into 6 tetrahedra per cube along its main diagonal (Freudenthal-Kuhn
    split, conforming across cubes); interior nodes moved by up to
    perturb * h per axis; with shuffle, node numbers, element numbers and the
    corner order of every element are permuted at random, so nothing about
    the numbering is structured.  Returns X [n, 3] float64, tets [E, 4] int32."""
    if isinstance(N, int):
        N = (N, N, N)
    Nx, Ny, Nz = N
    g = rng(seed)
    ax = [np.linspace(lo[d], hi[d], N[d] + 1) for d in range(3)]
    Z, Y, Xc = np.meshgrid(ax[2], ax[1], ax[0], indexing="ij")
    X = np.stack([Xc.ravel(), Y.ravel(), Z.ravel()], axis=1)
    h = np.array([(hi[d] - lo[d]) / N[d] for d in range(3)])
    if perturb:
        inner = np.all((X > np.array(lo) + 1e-12) & (X < np.array(hi) - 1e-12), axis=1)
        X[inner] += perturb * g.uniform(-1, 1, (int(inner.sum()), 3)) * h[None, :]

    perms = np.array([(0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)])
    # corner offsets of the 6 tetrahedra: the path 0 -> e_p0 -> e_p0 + e_p1 -> (1,1,1)
    off = np.zeros((6, 4, 3), dtype=np.int64)
    for t, p in enumerate(perms):
        c = np.zeros(3, dtype=np.int64)
        for s_, d in enumerate(p):
            c[d] = 1
            off[t, s_ + 1] = c
    k, j, i = np.meshgrid(np.arange(Nz), np.arange(Ny), np.arange(Nx), indexing="ij")
    base = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)           # cubes, x fastest
    corner = base[:, None, None, :] + off[None, :, :, :]                   # [cubes, 6, 4, 3]
    tets = (corner[..., 0] + (Nx + 1) * (corner[..., 1] + (Ny + 1) * corner[..., 2])).reshape(-1, 4)
    if shuffle:
        n = X.shape[0]
        new_of_old = g.permutation(n)
        Xs = np.empty_like(X)
        Xs[new_of_old] = X
        X = Xs
        tets = new_of_old[tets]
        tets = tets[g.permutation(len(tets))]
        rot = g.integers(0, 4, len(tets))
        tets = tets[np.arange(len(tets))[:, None], (np.arange(4)[None, :] - rot[:, None]) % 4]
    return X, tets.astype(np.int32)
