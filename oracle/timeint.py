"""Generalized-alpha time integration constants and stage values (Sec. 2.4).

TEST INFRASTRUCTURE ONLY (see the package docstring).

The paper integrates in time with the generalized-alpha method of Chung and
Hulbert / Jansen et al. in the variant of Liu et al. 2021 that evaluates the
pressure at t_{n+1}.  With spectral radius rho_inf:

  alpha_m = (3 - rho_inf) / (2 (1 + rho_inf)),  alpha_f = 1 / (1 + rho_inf),
  gamma   = 1/2 + alpha_m - alpha_f;

  V_{n+1}      = V_n + dt Vdot_n + gamma dt (Vdot_{n+1} - Vdot_n)
  V_{n+af}     = V_n + alpha_f (V_{n+1} - V_n)
  Vdot_{n+am}  = Vdot_n + alpha_m (Vdot_{n+1} - Vdot_n)

The unknown is y = (Vdot_{n+1}, P_{n+1}); the stage handed to the residual is
U = (V_{n+af}, P_{n+1}) and A = (Vdot_{n+am}, s).  The chain factors of the
Jacobian are dA/dVdot_{n+1} = alpha_m and dU/dVdot_{n+1} = alpha_f gamma dt.

Pins: the constants at rho_inf = 0.5 (5/6, 2/3, 2/3) and rho_inf = 1 (the
trapezoidal rule 1/2, 1/2, 1/2); constant acceleration is integrated exactly.
"""
from __future__ import annotations

import numpy as np


def alphas(rho_inf: float):
    am = 0.5 * (3.0 - rho_inf) / (1.0 + rho_inf)
    af = 1.0 / (1.0 + rho_inf)
    gamma = 0.5 + am - af
    return am, af, gamma


def chain_factors(rho_inf: float, dt: float):
    am, af, gamma = alphas(rho_inf)
    return am, af * gamma * dt


def stage(y, Vn, An, dt, rho_inf, s=None):
    """Stage (U, A) from unknown y = [Vdot_{n+1} | P_{n+1}] and history.

    y, Vn, An are [n,4]; Vn[:, :3] = V_n, An[:, :3] = Vdot_n.  s (optional)
    fills A[:, 3]; otherwise A[:, 3] = 1.
    """
    am, af, gamma = alphas(rho_inf)
    y = np.asarray(y, dtype=np.float64)
    V1 = Vn[:, :3] + dt * An[:, :3] + gamma * dt * (y[:, :3] - An[:, :3])
    U = np.empty_like(y)
    A = np.empty_like(y)
    U[:, :3] = Vn[:, :3] + af * (V1 - Vn[:, :3])
    U[:, 3] = y[:, 3]
    A[:, :3] = An[:, :3] + am * (y[:, :3] - An[:, :3])
    A[:, 3] = 1.0 if s is None else s
    return U, A


def velocity_next(y, Vn, An, dt, rho_inf):
    """V_{n+1} for the unknown y."""
    _, _, gamma = alphas(rho_inf)
    return Vn[:, :3] + dt * An[:, :3] + gamma * dt * (y[:, :3] - An[:, :3])
