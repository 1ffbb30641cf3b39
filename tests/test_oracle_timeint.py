"""Pins of the generalized-alpha constants and stage values (Sec. 2.4)."""
import numpy as np
import pytest


def test_alpha_constants(oracle):
    ti = oracle.timeint
    am, af, g = ti.alphas(0.5)
    assert (am, af, g) == pytest.approx((5 / 6, 2 / 3, 2 / 3), abs=1e-15)
    # rho_inf = 1: no numerical damping, the trapezoidal rule
    assert ti.alphas(1.0) == pytest.approx((0.5, 0.5, 0.5), abs=1e-15)
    # rho_inf = 0: asymptotic annihilation, gamma = 1
    assert ti.alphas(0.0) == pytest.approx((1.5, 1.0, 1.0), abs=1e-15)
    # second order accuracy condition of Jansen et al.: gamma = 1/2 + am - af
    for r in np.linspace(0, 1, 7):
        am, af, g = ti.alphas(r)
        assert g == pytest.approx(0.5 + am - af)


def test_constant_acceleration_is_exact(oracle):
    """With Vdot_n = Vdot_{n+1} = a the update is V_{n+1} = V_n + dt a."""
    ti = oracle.timeint
    rng = np.random.default_rng(0)
    n, dt = 10, 0.01
    a = rng.normal(size=(n, 4))
    Vn = rng.normal(size=(n, 4))
    for r in (0.0, 0.5, 1.0):
        V1 = ti.velocity_next(a, Vn, a, dt, r)
        assert np.abs(V1 - (Vn[:, :3] + dt * a[:, :3])).max() < 1e-15
        U, A = ti.stage(a, Vn, a, dt, r)
        am, af, _ = ti.alphas(r)
        assert np.abs(A[:, :3] - a[:, :3]).max() < 1e-15
        assert np.abs(U[:, :3] - (Vn[:, :3] + af * dt * a[:, :3])).max() < 1e-15
        assert np.array_equal(U[:, 3], a[:, 3])


def test_chain_factors_match_stage_derivative(oracle):
    ti = oracle.timeint
    rng = np.random.default_rng(1)
    n, dt, r = 5, 0.003, 0.5
    y, Vn, An = rng.normal(size=(n, 4)), rng.normal(size=(n, 4)), rng.normal(size=(n, 4))
    dy = np.zeros((n, 4))
    dy[:, :3] = rng.normal(size=(n, 3))
    U0, A0 = ti.stage(y, Vn, An, dt, r)
    U1, A1 = ti.stage(y + dy, Vn, An, dt, r)
    c_a, c_v = ti.chain_factors(r, dt)
    assert np.abs((A1 - A0)[:, :3] - c_a * dy[:, :3]).max() < 1e-14
    assert np.abs((U1 - U0)[:, :3] - c_v * dy[:, :3]).max() < 1e-15
