"""FP64 reference of the learned initial guess (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The network predicts, per node, the increment of the unknown over a time step,
y_{n+1} - y_n, used as the Newton predictor y^(0) = y_n + dy_hat.  Inputs per
node (112): the 27-node stencil (offsets -1..1 per axis, zero-padded outside
the grid) of the velocity V_n (3) and pressure P_n (1), then the node's
extrapolated increment e = 2 d_{n-1} - d_{n-2} (4), where d_k = y_{k+1} - y_k.
Output (4): the correction c with dy_hat = e + c.  Features and targets are
normalised per channel: x_hat = (x - mean_x) / std_x, c = mean_c + std_c * o.

Network: o = W3^T relu(W2^T relu(W1^T x_hat + b1) + b2) + b3 with W1 [112,256],
W2 [256,256], W3 [256,4] (row = input), loss = (1/B) sum_rows 1/2 |o - t|^2.
Adam with bias correction.

Pins (tests/test_oracle_mlp.py): central-difference gradient check of the
backward pass; the stencil features against direct indexing on a tiny grid;
Adam against its closed form; the BF16 rounding against its definition
(exact on representable values, nearest neighbour otherwise, ties to even).
"""
from __future__ import annotations

import numpy as np

N_IN, N_H, N_OUT = 112, 256, 4
STENCIL = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def param_shapes():
    return [("W1", (N_IN, N_H)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)),
            ("W3", (N_H, N_OUT)), ("b3", (N_OUT,))]


def n_params():
    return sum(int(np.prod(s)) for _, s in param_shapes())


def unflatten(theta):
    out, k = {}, 0
    for name, shp in param_shapes():
        sz = int(np.prod(shp))
        out[name] = np.asarray(theta[k:k + sz], dtype=np.float64).reshape(shp)
        k += sz
    return out


def flatten(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).ravel()
                           for name, _ in param_shapes()])


def features(N, V, P, d1, d2, idx=None):
    """Raw (unnormalised) features [k, 112] of the nodes idx (all if None).

    V [n,3] velocity, P [n] pressure, d1, d2 [n,4] the last two increments.
    """
    if np.isscalar(N):
        N = (N, N, N)
    nx, ny, nz = N[0] + 1, N[1] + 1, N[2] + 1
    n = nx * ny * nz
    idx = np.arange(n) if idx is None else np.asarray(idx)
    i, j, k = idx % nx, (idx // nx) % ny, idx // (nx * ny)
    F = np.zeros((len(idx), N_IN))
    for s, (dx, dy, dz) in enumerate(STENCIL):
        ii, jj, kk = i + dx, j + dy, k + dz
        ok = (ii >= 0) & (ii < nx) & (jj >= 0) & (jj < ny) & (kk >= 0) & (kk < nz)
        nb = np.where(ok, ii + nx * (jj + ny * kk), 0)
        F[:, 4 * s:4 * s + 3] = np.where(ok[:, None], V[nb, :3], 0.0)
        F[:, 4 * s + 3] = np.where(ok, P[nb], 0.0)
    F[:, 108:112] = 2.0 * d1[idx] - d2[idx]
    return F


def round_bf16(a):
    """Round to the nearest bfloat16 (ties to even), via float32, back to FP64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _mm(A, B, bf16):
    """Matrix product; with bf16=True both operands are first rounded to FP32
    and then to BF16, as the tensor-core path does, and accumulated exactly."""
    if bf16:
        return round_bf16(A) @ round_bf16(B)
    return A @ B


def forward(p, X, bf16=False):
    f32 = (lambda a: a.astype(np.float32).astype(np.float64)) if bf16 else (lambda a: a)
    Z1 = f32(_mm(X, p["W1"], bf16) + p["b1"])
    H1 = np.maximum(Z1, 0.0)
    Z2 = f32(_mm(H1, p["W2"], bf16) + p["b2"])
    H2 = np.maximum(Z2, 0.0)
    O = f32(_mm(H2, p["W3"], bf16) + p["b3"])
    return O, (X, Z1, H1, Z2, H2)


def loss_and_grad(p, X, T, bf16=False):
    """Loss (1/B) sum 1/2 |O - T|^2 and its gradient w.r.t. every parameter.

    bf16=True reproduces the operand rounding of the tensor-core kernels (a
    statement of what that path computes, not of the network's definition).
    """
    B = X.shape[0]
    f32 = (lambda a: a.astype(np.float32).astype(np.float64)) if bf16 else (lambda a: a)
    O, (X, Z1, H1, Z2, H2) = forward(p, X, bf16)
    dO = f32((O - T) / B)
    loss = 0.5 * np.sum((O - T) ** 2) / B
    g = {}
    g["W3"] = _mm(H2.T, dO, bf16)
    g["b3"] = dO.sum(axis=0)
    dZ2 = f32(_mm(dO, p["W3"].T, bf16)) * (Z2 > 0)
    g["W2"] = _mm(H1.T, dZ2, bf16)
    g["b2"] = dZ2.sum(axis=0)
    dZ1 = f32(_mm(dZ2, p["W2"].T, bf16)) * (Z1 > 0)
    g["W1"] = _mm(X.T, dZ1, bf16)
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def adam(theta, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (t counts from 1); returns new (theta, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def init_params(seed):
    """He-style initialisation from a seed (FP64; the GPU side rounds to FP32)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in param_shapes():
        if name.startswith("W"):
            p[name] = rng.normal(scale=np.sqrt(2.0 / shp[0]), size=shp)
        else:
            p[name] = np.zeros(shp)
    return p
