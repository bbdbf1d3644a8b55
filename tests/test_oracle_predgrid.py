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


def test_r23_truncation_closed_forms():
    """trunc_f32 (R23's single-precision origin): exact for values that are
    floats, toward zero for others (unlike round-to-nearest), signed zero
    below the normal float range, signed infinity above it, NaN kept."""
    two = 2.0
    x = np.array([0.75, -3.5, 1 + two ** -30, 1 + two ** -23 - two ** -30,
                  -(1 + two ** -23 + two ** -30), 1e-300, -1e-300, 1e300, -1e300,
                  np.inf, -np.inf, np.nan, 0.0, -0.0, two ** -126, two ** 127 * 1.5])
    t = oracle.trunc_f32(x)
    assert t.dtype == np.float32
    want = np.array([0.75, -3.5, 1.0, 1.0, -(1 + two ** -23), 0.0, -0.0, np.inf, -np.inf,
                     np.inf, -np.inf, np.nan, 0.0, -0.0, two ** -126, two ** 127 * 1.5],
                    dtype=np.float32)
    assert np.array_equal(t, want, equal_nan=True)
    assert np.array_equal(np.signbit(t), np.signbit(want))
    # round to nearest would have given 1 + 2^-23 for the fourth value
    assert np.float32(x[3]) == np.float32(1 + two ** -23)


def test_r23_cells_closed_forms():
    """cell_f32: floor((v - lo) * inv) in float32, clamped; NaN and negative
    quotients give cell 0, +inf the last cell."""
    v = np.array([0.5, 2.5, 9.99, 10.0, 123.0, -0.1, -0.0, np.nan, np.inf, -np.inf],
                 dtype=np.float32)
    c = oracle.cell_f32(v, 0.0, 1.0, 10)
    assert c.tolist() == [0, 2, 9, 9, 9, 0, 0, 0, 9, 0]
    # with a cell size of 1/4 and origin 1: (v - 1) * 4
    c = oracle.cell_f32(np.array([1.0, 1.24, 1.25, 2.0], dtype=np.float32), 1.0, 4.0, 100)
    assert c.tolist() == [0, 0, 1, 4]


def test_r23_origin_agrees_with_fp64_away_from_faces():
    """Away from cell faces the single-precision origin selects the same
    predictor cell and the same ASG cell as the FP64 formula (its rounding
    error is ~1e-7 of the box; cells are ~1e-2 here)."""
    c = make_case("tg2d", n_side=41)
    om = oracle.Mesh(c.xyz, c.conn, grid=40, pred_stride=3)
    rng = np.random.default_rng(3)
    dhat = rng.uniform(-3, 3, size=(int(np.prod(om.pgrid)), 2)).astype(np.float32)
    pc, ac = om.cnn_origin_cells(c.x, dhat)
    y = c.x + dhat[om.pred_cells(c.x)].astype(np.float64) * om.ps
    s = (om.hi - om.lo) / om.grid
    fx = (c.x - om.lo) / om.ps
    fy = (y - om.lo) / s
    far = ((np.abs(fx - np.round(fx)) > 1e-4).all(axis=1)
           & (np.abs(fy - np.round(fy)) > 1e-4).all(axis=1))
    assert far.mean() > 0.9
    assert np.array_equal(pc[far], om.pred_cells(c.x)[far])
    assert np.array_equal(ac[far], om.cells(y)[far])
