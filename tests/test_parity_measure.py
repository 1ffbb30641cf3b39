"""The local parity measure (tests/parity.py) on planted errors, on the CPU.

Each case plants an error that a single norm over the whole array lets pass
at the FP32 tolerance and checks that the local measure rejects it; a
correct array with rounding-level noise passes.
"""
import numpy as np

import parity

TOL = 1e-5


def global_rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def field(N, seed=0):
    n = (N + 1) ** 3
    rng = np.random.default_rng(seed)
    R = np.empty((n, 4))
    R[:, :3] = rng.normal(size=(n, 3))
    R[:, 3] = 1e-3 * rng.normal(size=n)    # continuity rows much smaller
    return R


def test_boundary_mask_counts():
    for N in [(1, 1, 1), (4, 3, 5), (8, 8, 8)]:
        b = parity.boundary_mask(N)
        n = np.prod(np.array(N) + 1)
        inner = np.prod(np.array(N) - 1)
        assert len(b) == n and (~b).sum() == inner
    b = parity.boundary_mask((3, 2, 2)).reshape(3, 3, 4)   # [z][y][x]
    assert b[:, :, 0].all() and b[:, :, 3].all() and b[0].all() and b[2].all()
    assert not b[1, 1, 1] and not b[1, 1, 2]


def test_rounding_noise_passes():
    R = field(16)
    got = R * (1 + 1e-7 * np.random.default_rng(1).normal(size=R.shape))
    assert parity.rel_local(got, R, (16, 16, 16)) < TOL


def test_wrong_continuity_row_is_caught():
    R = field(16)
    got = R.copy()
    got[:, 3] *= 1.01                       # 1 % off in the small row only
    assert global_rel(got, R) < TOL
    err, part = parity.worst(got, R, (16, 16, 16))
    assert err > TOL and part[0] == "continuity"


def test_wrong_face_is_caught():
    N = 32
    R = field(N)
    got = R.copy()
    face = np.arange(len(R)).reshape(N + 1, N + 1, N + 1)[:, :, 0].ravel()   # x = 0
    got[face, :3] += 5e-5 * R[face, :3]
    assert global_rel(got, R) < TOL
    err, part = parity.worst(got, R, (N, N, N))
    assert err > TOL and part[1] == "boundary"


def test_few_wrong_entries_are_caught():
    R = field(32)
    got = R.copy()
    got[::5000, 1] += 3e-4                  # 8 entries of 143,748 x 3
    assert global_rel(got, R) < TOL
    assert parity.rel_local(got, R) > TOL


def test_point_arrays_and_zero_parts():
    u = np.random.default_rng(3).normal(size=(1000, 3))
    u[:100] = 0.0                           # outside points interpolate to 0
    assert parity.rel_local(u.copy(), u) == 0.0
    bad = u.copy()
    bad[:100] = 1e-3                        # non-zero where the reference is zero
    assert parity.rel_local(bad, u) > TOL
    assert parity.rel_local(np.zeros((0, 3)), np.zeros((0, 3))) == 0.0
