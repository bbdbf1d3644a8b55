"""Non-convex domain: the unit square with a disc taken out.

A walk of Algorithm 1 that meets the hole's boundary stops at a face with no
neighbour although the departure point may lie in the domain beyond it; the
exact search then finds the host (status FOUND_VIA_FALLBACK). These pins
check the oracle's exact location on such a mesh against brute force and
against the geometry of the hole.
"""

import numpy as np

import oracle
from workloads import make_case
from workloads.meshes import mesh_2d_hole


def test_hole_mesh_is_valid_and_has_the_hole():
    xyz, conn, h = mesh_2d_hole(41, 0.15)
    p = xyz[conn]
    area2 = ((p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) -
             (p[:, 1, 1] - p[:, 0, 1]) * (p[:, 2, 0] - p[:, 0, 0]))
    assert (area2 > 0).all()
    assert np.array_equal(np.unique(conn), np.arange(xyz.shape[0]))
    # covered area = square minus the polygon inscribed in the circle
    m = max(8, int(np.ceil(2 * np.pi * 0.15 / h)))
    poly = 0.5 * m * 0.15 ** 2 * np.sin(2 * np.pi / m)
    assert abs(0.5 * area2.sum() - (1.0 - poly)) < 1e-12


def test_exact_location_against_brute_force_and_the_hole():
    xyz, conn, h = mesh_2d_hole(41, 0.15)
    om = oracle.Mesh(xyz, conn, brute_limit=0)            # bucketed search
    rng = np.random.default_rng(3)
    pts = rng.random((4000, 2)) * 1.1 - 0.05
    got = om.locate(pts)
    v0, M = oracle.inverse_affine(xyz, conn)
    ref = oracle.locate_bruteforce(v0, M, pts, oracle.EPS)
    assert np.array_equal(got, ref)
    r = np.linalg.norm(pts - 0.5, axis=1)
    inside_square = (pts >= 0).all(axis=1) & (pts <= 1).all(axis=1)
    # well inside the hole or outside the square: no host
    assert (got[(r < 0.15 * np.cos(np.pi / 8) - 1e-9) | ~inside_square] == -1).all()
    # well inside the domain: a host
    assert (got[inside_square & (r > 0.15 + 1e-9)] >= 0).all()


def test_walks_blocked_by_the_hole_end_in_the_exact_search():
    c = make_case("hole2d", n_side=61)
    om = oracle.Mesh(c.xyz, c.conn)
    r = om.track(c.x, c.u, c.dt, mode="sns")
    blocked = r["reason"] == oracle.BOUNDARY
    # every walk that met a boundary is resolved by the exact search: found
    # beyond the hole (FOUND_VIA_FALLBACK) or outside the domain (OUTSIDE)
    assert np.array_equal(r["status"][blocked] == oracle.ST_FALLBACK, r["host"][blocked] >= 0)
    assert (r["status"] == oracle.ST_FALLBACK).sum() > 20
    assert (r["status"][~blocked] == oracle.ST_FOUND).all()


# --- 3-D: the cube with a ball taken out (the flow past a sphere, Sec. 3.2) --

def test_sphere_mesh_is_valid_and_has_the_ball():
    """Every tetrahedron keeps a non-zero volume, every vertex is used, the
    volume is the cube's minus exactly the dropped tetrahedra, and no
    remaining tetrahedron has its centroid in the ball."""
    from workloads.meshes import mesh_3d_sphere, mesh_3d
    xyz, conn, h = mesh_3d_sphere(17, 0.25)
    full_xyz, full_conn, _ = mesh_3d(17, 0.1, 11)
    def vol(x, c):
        a = x[c[:, 1]] - x[c[:, 0]]
        b = x[c[:, 2]] - x[c[:, 0]]
        d = x[c[:, 3]] - x[c[:, 0]]
        return np.einsum("ij,ij->i", a, np.cross(b, d)) / 6.0
    v = vol(xyz, conn)
    assert (np.abs(v) > 0).all()
    assert np.array_equal(np.unique(conn), np.arange(xyz.shape[0]))
    assert np.linalg.norm(xyz[conn].mean(axis=1) - 0.5, axis=1).min() > 0.25
    vf = vol(full_xyz, full_conn)
    cen = full_xyz[full_conn].mean(axis=1)
    dropped = np.linalg.norm(cen - 0.5, axis=1) <= 0.25
    assert abs(np.abs(vf).sum() - 1.0) < 1e-12
    assert abs(np.abs(v).sum() - (1.0 - np.abs(vf[dropped]).sum())) < 1e-12
    assert dropped.sum() > 100


def test_sphere_exact_location_against_brute_force_and_the_ball():
    from workloads.meshes import mesh_3d_sphere
    xyz, conn, h = mesh_3d_sphere(17, 0.25)
    om = oracle.Mesh(xyz, conn, brute_limit=0)            # bucketed search
    rng = np.random.default_rng(4)
    pts = rng.random((4000, 3)) * 1.1 - 0.05
    got = om.locate(pts)
    v0, M = oracle.inverse_affine(xyz, conn)
    ref = oracle.locate_bruteforce(v0, M, pts, oracle.EPS)
    assert np.array_equal(got, ref)
    r = np.linalg.norm(pts - 0.5, axis=1)
    inside_cube = (pts >= 0).all(axis=1) & (pts <= 1).all(axis=1)
    # a tetrahedron is dropped only if its centroid is in the ball, so its
    # points lie within radius + (its size, < 2h) of the centre; one kept has
    # its centroid outside, so it covers no point deeper than radius - 2h
    assert (got[(r < 0.25 - 2 * h) | ~inside_cube] == -1).all()
    assert (got[inside_cube & (r > 0.25 + 2 * h)] >= 0).all()


def test_sphere_walks_blocked_by_the_ball_end_in_the_exact_search():
    c = make_case("sphere3d", n_side=21)
    om = oracle.Mesh(c.xyz, c.conn)
    r = om.track(c.x, c.u, c.dt, mode="sns")
    blocked = r["reason"] == oracle.BOUNDARY
    assert np.array_equal(r["status"][blocked] == oracle.ST_FALLBACK, r["host"][blocked] >= 0)
    assert (r["status"] == oracle.ST_FALLBACK).sum() > 20
    assert (r["status"][~blocked] == oracle.ST_FOUND).all()
