"""Pins of the oracle's predictor grid (cells of p^d ASG cells, p odd).

The predictor grid is a coarser sampling of the ASG grid (Sec. 2.3: the ASG
pools several elements into each Cartesian cell). Checked against the ASG
grid routines of the C oracle, which it must reduce to for p = 1, and
against the index arithmetic of the definition for p = 3.
"""

import numpy as np
import pytest

import oracle
from workloads import make_case


@pytest.fixture(scope="module")
def meshes():
    c2 = make_case("tg2d", n_side=31)
    c3 = make_case("abc3d", n_side=9)
    return [(c2, oracle.Mesh(c2.xyz, c2.conn)), (c3, oracle.Mesh(c3.xyz, c3.conn))]


def _points(om, n, seed):
    rng = np.random.default_rng(seed)
    ext = om.hi - om.lo
    pts = om.lo - 0.1 * ext + rng.random((n, om.dim)) * 1.2 * ext
    pts[0] = np.nan
    pts[1] = om.hi
    pts[2] = om.lo
    return pts


def test_stride_one_is_the_asg_grid(meshes):
    for c, om in meshes:
        om.set_pred_stride(1)
        assert np.array_equal(om.pgrid, om.grid)
        pts = _points(om, 2000, 1)
        assert np.array_equal(om.pred_cells(pts), om.cells(pts))
        assert np.array_equal(om.pred_centres(), oracle.grid_centres(om.lo, om.hi, om.grid))


def test_stride_three_centres_are_middle_asg_centres(meshes):
    for c, om in meshes:
        om.set_pred_stride(3)
        assert np.array_equal(om.pgrid, om.grid // 3)
        fine = oracle.grid_centres(om.lo, om.hi, om.grid)
        pc = om.pred_centres()
        # predictor cell I <-> ASG cell 3 I + 1 on every axis
        idx = np.indices(tuple(om.pgrid[::-1])).reshape(om.dim, -1)[::-1]   # x fastest
        f = np.zeros(pc.shape[0], dtype=np.int64)
        for k in range(om.dim - 1, -1, -1):
            f = f * int(om.grid[k]) + 3 * idx[k] + 1
        assert np.abs(pc - fine[f]).max() <= 8 * np.finfo(float).eps * np.abs(fine).max()
        # each predictor centre lies in its own cell
        assert np.array_equal(om.pred_cells(pc), np.arange(pc.shape[0]))
        om.set_pred_stride(1)


def test_stride_three_cell_of_every_asg_centre(meshes):
    for c, om in meshes:
        om.set_pred_stride(3)
        fine = oracle.grid_centres(om.lo, om.hi, om.grid)
        idx = np.indices(tuple(om.grid[::-1])).reshape(om.dim, -1)[::-1]
        want = np.zeros(fine.shape[0], dtype=np.int64)
        for k in range(om.dim - 1, -1, -1):
            # ASG cells past the last whole predictor cell belong to it
            want = want * int(om.pgrid[k]) + np.minimum(idx[k] // 3, om.pgrid[k] - 1)
        assert np.array_equal(om.pred_cells(fine), want)
        # points outside the box clamp to the boundary cells, NaN to cell 0
        pts = _points(om, 500, 2)
        got = om.pred_cells(pts)
        assert got[0] == 0 and got.min() >= 0 and got.max() < np.prod(om.pgrid)
        om.set_pred_stride(1)


def test_even_stride_rejected(meshes):
    om = meshes[0][1]
    for p in (0, 2, 4, -1):
        with pytest.raises(ValueError):
            om.set_pred_stride(p)
