"""Pins of the FP64 reference of the learned initial guess."""
import numpy as np


def test_backward_matches_central_differences():
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = mlp.init_params(1)
    for k in p:
        if k.startswith("b"):
            p[k] = rng.normal(scale=0.1, size=p[k].shape)
    X = rng.normal(size=(7, mlp.N_IN))
    T = rng.normal(size=(7, mlp.N_OUT))
    loss, g = mlp.loss_and_grad(p, X, T)
    theta = mlp.flatten(p)
    gvec = mlp.flatten(g)
    # random directional derivatives plus a few coordinates of every tensor
    for trial in range(6):
        d = rng.normal(size=theta.shape)
        eps = 1e-6
        lp, _ = mlp.loss_and_grad(mlp.unflatten(theta + eps * d), X, T)
        lm, _ = mlp.loss_and_grad(mlp.unflatten(theta - eps * d), X, T)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - gvec @ d) <= 1e-6 * max(1.0, abs(fd))
    off = 0
    for name, shp in mlp.param_shapes():
        sz = int(np.prod(shp))
        for q in rng.integers(0, sz, size=3):
            e = np.zeros_like(theta)
            e[off + q] = 1.0
            lp, _ = mlp.loss_and_grad(mlp.unflatten(theta + 1e-6 * e), X, T)
            lm, _ = mlp.loss_and_grad(mlp.unflatten(theta - 1e-6 * e), X, T)
            assert abs((lp - lm) / 2e-6 - gvec[off + q]) < 1e-7, name
        off += sz


def test_features_are_the_padded_stencil():
    from oracle import mlp
    N = (3, 2, 4)
    n = 4 * 3 * 5
    rng = np.random.default_rng(3)
    V, P = rng.normal(size=(n, 3)), rng.normal(size=n)
    d1, d2 = rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    F = mlp.features(N, V, P, d1, d2)
    grid = np.arange(n).reshape(5, 3, 4)   # [k][j][i]
    for node in (0, 7, 23, n - 1):
        i, j, k = node % 4, (node // 4) % 3, node // 12
        col = 0
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    ii, jj, kk = i + dx, j + dy, k + dz
                    if 0 <= ii < 4 and 0 <= jj < 3 and 0 <= kk < 5:
                        nb = grid[kk, jj, ii]
                        want = np.concatenate([V[nb], [P[nb]]])
                    else:
                        want = np.zeros(4)
                    assert np.array_equal(F[node, col:col + 4], want)
                    col += 4
        assert np.array_equal(F[node, 108:], 2 * d1[node] - d2[node])


def test_adam_closed_form_first_step():
    """First Adam step moves every coordinate by lr * sign(g) (bias-corrected)."""
    from oracle import mlp
    theta = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 1e-3])
    th, m, v = mlp.adam(theta, g, np.zeros(3), np.zeros(3), 1, lr=0.01, eps=0.0)
    assert np.allclose(th, theta - 0.01 * np.sign(g), rtol=0, atol=1e-15)


def test_bf16_rounding_definition():
    from oracle import mlp
    # representable values are unchanged
    v = np.array([1.0, -2.5, 0.15625, 3.0 * 2.0 ** -20, 65280.0])
    assert np.array_equal(mlp.round_bf16(v), v)
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7: ties to even (1.0)
    assert mlp.round_bf16(np.array([1.0 + 2.0 ** -8]))[0] == 1.0
    # 1 + 3*2^-8 is halfway between 1+2^-7 and 1+2^-6: ties to even (1 + 2^-6)
    assert mlp.round_bf16(np.array([1.0 + 3 * 2.0 ** -8]))[0] == 1.0 + 2.0 ** -6
    # otherwise the nearest BF16 value (8 significant bits)
    x = np.random.default_rng(0).normal(size=1000)
    r = mlp.round_bf16(x)
    e = np.floor(np.log2(np.abs(x)))
    assert np.all(np.abs(r - x) <= 2.0 ** (e - 8) * (1 + 1e-12))
    assert np.all(np.abs(r * 2.0 ** (7 - e) - np.round(r * 2.0 ** (7 - e))) == 0)
