"""Pins of the interface scaling field oracle (Sec. 2.1)."""
import numpy as np
import pytest

from oracle import core
from oracle import interface as itf


def test_one_point_marks_its_cell_or_the_dilated_block():
    g = core.Grid((6, 5, 7))
    X = np.array([[0.45, 0.5, 0.5]])                      # cell (2, 2, 3)
    e, _, _ = core.locate(g, X)
    s0 = itf.scaling_field(g, e, 50.0, 0).reshape(8, 6, 7)
    assert set(np.unique(s0)) == {1.0, 50.0}
    assert np.count_nonzero(s0 == 50.0) == 8
    assert np.all(s0[3:5, 2:4, 2:4] == 50.0)
    s1 = itf.scaling_field(g, e, 50.0, 1).reshape(8, 6, 7)
    assert np.count_nonzero(s1 == 50.0) == 4 ** 3
    assert np.all(s1[2:6, 1:5, 1:5] == 50.0)


def test_band_is_clipped_at_the_grid_boundary():
    g = core.Grid(4)
    e, _, _ = core.locate(g, np.array([[0.01, 0.01, 0.99]]))   # corner cell (0, 0, 3)
    s = itf.scaling_field(g, e, 10.0, 2).reshape(5, 5, 5)
    # cells x, y in 0..2 and z in 1..3 -> nodes x, y in 0..3 and z in 1..4
    assert np.count_nonzero(s == 10.0) == 4 * 4 * 4
    assert np.all(s[1:5, 0:4, 0:4] == 10.0)


def test_band_of_a_set_is_the_union_and_outside_points_are_ignored():
    g = core.Grid((8, 8, 8))
    rng = np.random.default_rng(0)
    X = np.concatenate([rng.uniform(0, 1, (20, 3)), [[2.0, 0.5, 0.5]]])
    e, _, nout = core.locate(g, X)
    assert nout == 1
    for layers in (0, 1):
        s_all = itf.scaling_field(g, e, 7.0, layers)
        union = np.zeros(g.n_nodes, dtype=bool)
        for b in range(X.shape[0]):
            union |= itf.scaling_field(g, e[b:b + 1], 7.0, layers) == 7.0
        assert np.array_equal(s_all == 7.0, union)


def test_no_points_gives_ones():
    g = core.Grid(3)
    s = itf.scaling_field(g, np.zeros(0, dtype=np.int32), 100.0, 1)
    assert np.all(s == 1.0) and s.shape == (64,)
