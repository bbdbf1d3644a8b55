"""Seeded mesh generators (inputs only).

2-D: an n x n lattice on the unit square, interior points jittered uniformly
by +-j*h per coordinate (boundary points fixed), Delaunay-triangulated with
scipy's Qhull. 3-D: an n^3 lattice on the unit cube, interior points jittered
by +-j*h, each lattice cell split into six Kuhn tetrahedra along its main
diagonal; a vertex whose jitter inverts one of its tetrahedra is redrawn.

Connectivity rows keep the vertex order the generator produces; the method
never reorders the vertices of an element, so local index i always names the
same vertex on both sides.
"""

import functools

import numpy as np


def lattice_2d(n_side, jitter, seed):
    """Jittered n_side x n_side lattice on [0,1]^2; returns (xyz[n_v,2], h)."""
    h = 1.0 / (n_side - 1)
    g = np.linspace(0.0, 1.0, n_side)
    X, Y = np.meshgrid(g, g, indexing="xy")          # node id = iy*n + ix
    p = np.stack([X.ravel(), Y.ravel()], axis=1)
    rng = np.random.default_rng(seed)
    dj = rng.uniform(-jitter * h, jitter * h, size=p.shape)
    i = np.arange(n_side)
    ix = np.tile(i, n_side)
    iy = np.repeat(i, n_side)
    edge = (ix == 0) | (ix == n_side - 1) | (iy == 0) | (iy == n_side - 1)
    dj[edge] = 0.0
    return np.ascontiguousarray(p + dj), h


def delaunay_2d(xyz):
    """Delaunay triangulation of a 2-D point set; conn[n_e,3] int32."""
    from scipy.spatial import Delaunay
    tri = Delaunay(xyz)
    if len(tri.coplanar):
        raise RuntimeError("Qhull dropped %d coplanar points" % len(tri.coplanar))
    return np.ascontiguousarray(tri.simplices.astype(np.int32))


@functools.lru_cache(maxsize=8)
def _mesh_2d_cached(n_side, jitter, seed):
    xyz, h = lattice_2d(n_side, jitter, seed)
    conn = delaunay_2d(xyz)
    xyz.setflags(write=False)
    conn.setflags(write=False)
    return xyz, conn, h


def mesh_2d(n_side, jitter=0.3, seed=1):
    """(xyz, conn, h) of the jittered Delaunay square (read-only, cached)."""
    return _mesh_2d_cached(int(n_side), float(jitter), int(seed))


@functools.lru_cache(maxsize=4)
def _mesh_2d_hole_cached(n_side, radius, jitter, seed):
    xyz, h = lattice_2d(n_side, jitter, seed)
    c = np.array([0.5, 0.5])
    keep = np.linalg.norm(xyz - c, axis=1) > radius + 0.5 * h
    m = max(8, int(np.ceil(2 * np.pi * radius / h)))
    t = 2 * np.pi * np.arange(m) / m
    ring = c + radius * np.stack([np.cos(t), np.sin(t)], axis=1)
    pts = np.concatenate([xyz[keep], ring])
    conn = delaunay_2d(pts)
    cen = pts[conn].mean(axis=1)
    conn = conn[np.linalg.norm(cen - c, axis=1) > radius]
    used = np.unique(conn)                       # drop vertices no triangle uses
    remap = np.full(pts.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    pts = np.ascontiguousarray(pts[used])
    conn = np.ascontiguousarray(remap[conn].astype(np.int32))
    pts.setflags(write=False)
    conn.setflags(write=False)
    return pts, conn, h


def mesh_2d_hole(n_side, radius=0.2, jitter=0.3, seed=7):
    """(xyz, conn, h): the jittered Delaunay square with a disc of `radius`
    at its centre taken out (a non-convex domain: walks can meet the hole's
    boundary while the departure point lies in the domain beyond it). The
    lattice points within radius + h/2 of the centre are replaced by a ring of
    points on the circle, spaced about h; triangles whose centroid lies in the
    disc are dropped (read-only, cached)."""
    return _mesh_2d_hole_cached(int(n_side), float(radius), float(jitter), int(seed))


# Six Kuhn tetrahedra of the cell [0,1]^3: each is the path
# 000 -> e_a -> e_a+e_b -> 111 for one permutation (a, b, c) of the axes.
# Corner bit k of a corner index is its offset along axis k.
def _kuhn_corners():
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c0 = 0
        c1 = c0 | (1 << perm[0])
        c2 = c1 | (1 << perm[1])
        c3 = 7
        tets.append((c0, c1, c2, c3))
    return np.array(tets, dtype=np.int64)


def _signed_volumes(xyz, conn):
    a = xyz[conn[:, 1]] - xyz[conn[:, 0]]
    b = xyz[conn[:, 2]] - xyz[conn[:, 0]]
    c = xyz[conn[:, 3]] - xyz[conn[:, 0]]
    return np.einsum("ij,ij->i", a, np.cross(b, c))


def kuhn_3d(n_side, jitter, seed, max_redraw=64):
    """Jittered unit cube split into 6 Kuhn tets per cell.

    Returns (xyz[n_v,3], conn[n_e,4] int32, h); node id = (iz*n + iy)*n + ix.
    Every tetrahedron keeps the orientation it has on the unjittered lattice;
    vertices of a tetrahedron whose orientation flips (or collapses) are
    redrawn from the same generator.
    """
    n = n_side
    h = 1.0 / (n - 1)
    g = np.linspace(0.0, 1.0, n)
    Z, Y, X = np.meshgrid(g, g, g, indexing="ij")
    base = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    i = np.arange(n)
    ix = np.tile(i, n * n)
    iy = np.tile(np.repeat(i, n), n)
    iz = np.repeat(i, n * n)
    interior = (ix > 0) & (ix < n - 1) & (iy > 0) & (iy < n - 1) & (iz > 0) & (iz < n - 1)

    # connectivity
    c = np.arange(n - 1)
    cx = np.tile(c, (n - 1) ** 2)
    cy = np.tile(np.repeat(c, n - 1), n - 1)
    cz = np.repeat(c, (n - 1) ** 2)
    corner = np.empty((cx.size, 8), dtype=np.int64)
    for k in range(8):
        dx, dy, dz = k & 1, (k >> 1) & 1, (k >> 2) & 1
        corner[:, k] = ((cz + dz) * n + (cy + dy)) * n + (cx + dx)
    kc = _kuhn_corners()
    conn = corner[:, kc].reshape(-1, 4)
    ref_sign = np.sign(_signed_volumes(base, conn))

    rng = np.random.default_rng(seed)
    dj = rng.uniform(-jitter * h, jitter * h, size=base.shape)
    dj[~interior] = 0.0
    xyz = base + dj
    for _ in range(max_redraw):
        vol = _signed_volumes(xyz, conn)
        bad = np.sign(vol) != ref_sign
        if not bad.any():
            break
        verts = np.unique(conn[bad].ravel())
        verts = verts[interior[verts]]
        dj = rng.uniform(-jitter * h, jitter * h, size=(verts.size, 3))
        xyz[verts] = base[verts] + dj
    else:
        raise RuntimeError("could not draw a valid jittered Kuhn mesh")
    return np.ascontiguousarray(xyz), np.ascontiguousarray(conn.astype(np.int32)), h


@functools.lru_cache(maxsize=4)
def _mesh_3d_cached(n_side, jitter, seed):
    xyz, conn, h = kuhn_3d(n_side, jitter, seed)
    xyz.setflags(write=False)
    conn.setflags(write=False)
    return xyz, conn, h


def mesh_3d(n_side, jitter=0.1, seed=3):
    """(xyz, conn, h) of the jittered Kuhn cube (read-only, cached)."""
    return _mesh_3d_cached(int(n_side), float(jitter), int(seed))


def lattice_tris_2d(n_side, jitter, seed, max_redraw=64):
    """(xyz, conn, h): the unit square's n x n lattice, interior points jittered
    uniformly by up to jitter * h, each lattice square split along its
    rising diagonal into two triangles (a structured triangulation, fast at
    any size). Interior points of a triangle that would flip are redrawn."""
    xyz, h = lattice_2d(n_side, 0.0, seed)
    n = n_side
    i = np.arange(n - 1)
    ix = np.tile(i, n - 1)
    iy = np.repeat(i, n - 1)
    v00 = iy * n + ix
    v10, v01, v11 = v00 + 1, v00 + n, v00 + n + 1
    conn = np.concatenate([np.stack([v00, v10, v11], axis=1),
                           np.stack([v00, v11, v01], axis=1)]).astype(np.int32)
    base = xyz.copy()
    gx = np.tile(np.arange(n), n)
    gy = np.repeat(np.arange(n), n)
    interior = (gx > 0) & (gx < n - 1) & (gy > 0) & (gy < n - 1)
    rng = np.random.default_rng(seed)
    dj = rng.uniform(-jitter * h, jitter * h, size=base.shape)
    dj[~interior] = 0.0
    xyz = base + dj

    def area2(p):
        q = p[conn]
        return ((q[:, 1, 0] - q[:, 0, 0]) * (q[:, 2, 1] - q[:, 0, 1]) -
                (q[:, 1, 1] - q[:, 0, 1]) * (q[:, 2, 0] - q[:, 0, 0]))
    for _ in range(max_redraw):
        bad = area2(xyz) <= 0
        if not bad.any():
            break
        verts = np.unique(conn[bad].ravel())
        verts = verts[interior[verts]]
        xyz[verts] = base[verts] + rng.uniform(-jitter * h, jitter * h, size=(verts.size, 2))
    else:
        raise RuntimeError("could not draw a valid jittered lattice triangulation")
    return np.ascontiguousarray(xyz), np.ascontiguousarray(conn), h


def serving_mesh_sizes(seed=5):
    """The serving workload's 32 meshes: 16 triangle meshes with 0.1M-4M
    elements and 16 tetrahedral meshes with 0.5M-6M elements, sizes drawn
    log-uniformly (seeded). Returns [(dim, n_side)] with n_side the lattice
    points per axis that give about that many elements (2 (n-1)^2 triangles,
    6 (n-1)^3 tetrahedra)."""
    rng = np.random.default_rng(seed)
    out = []
    for dim, lo, hi in ((2, 1e5, 4e6), (3, 5e5, 6e6)):
        for ne in np.exp(rng.uniform(np.log(lo), np.log(hi), size=16)):
            per = 2.0 if dim == 2 else 6.0
            out.append((dim, int(round((ne / per) ** (1.0 / dim))) + 1))
    return out


@functools.lru_cache(maxsize=4)
def _mesh_3d_sphere_cached(n_side, radius, jitter, seed):
    xyz, conn, h = kuhn_3d(n_side, jitter, seed)
    c = np.array([0.5, 0.5, 0.5])
    cen = xyz[conn].mean(axis=1)
    conn = conn[np.linalg.norm(cen - c, axis=1) > radius]
    used = np.unique(conn)                       # drop vertices no tetrahedron uses
    remap = np.full(xyz.shape[0], -1, dtype=np.int64)
    remap[used] = np.arange(used.shape[0])
    xyz = np.ascontiguousarray(xyz[used])
    conn = np.ascontiguousarray(remap[conn].astype(np.int32))
    xyz.setflags(write=False)
    conn.setflags(write=False)
    return xyz, conn, h


def mesh_3d_sphere(n_side, radius=0.2, jitter=0.1, seed=11):
    """(xyz, conn, h): the jittered Kuhn cube with a ball of `radius` at its
    centre taken out, the obstacle of the flow past a sphere (a non-convex
    domain: walks can meet the ball's boundary while the departure point lies
    in the domain beyond it). Tetrahedra whose centroid lies in the ball are
    dropped, then the vertices no tetrahedron uses (read-only, cached)."""
    return _mesh_3d_sphere_cached(int(n_side), float(radius), float(jitter), int(seed))


def tie_meshes():
    """Two-element meshes in which the start element's smallest barycentric
    coordinates are exactly equal at the query point: element 0 is the unit
    simplex (v0 at the origin, so M is the identity and lambda_k = p_k for
    k >= 1, computed without rounding) and p has equal negative coordinates.
    Element 1 lies across exactly one face of element 0 and contains p; every
    other face of element 0 is on the boundary.

    Returns a list of (name, xyz, conn, p, face): `face` is the local face of
    element 0 that element 1 lies across."""
    out = []
    # 2-D, p = (-1/2, -1/2): lambda = (2, -1/2, -1/2)
    p2 = np.array([[-0.5, -0.5]])
    out.append(("2d-across-face-1",
                np.array([[0, 0], [1, 0], [0, 1], [-2, -3]], dtype=np.float64),
                np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32), p2, 1))
    out.append(("2d-across-face-2",
                np.array([[0, 0], [1, 0], [0, 1], [-3, -2]], dtype=np.float64),
                np.array([[0, 1, 2], [0, 3, 1]], dtype=np.int32), p2, 2))
    # 3-D, p = (-1/4, -1/4, -1/4): lambda = (7/4, -1/4, -1/4, -1/4)
    p3 = np.array([[-0.25, -0.25, -0.25]])
    unit = [[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]]
    out.append(("3d-across-face-1",
                np.array(unit + [[-3, -4, -4]], dtype=np.float64),
                np.array([[0, 1, 2, 3], [0, 3, 2, 4]], dtype=np.int32), p3, 1))
    out.append(("3d-across-face-3",
                np.array(unit + [[-4, -4, -3]], dtype=np.float64),
                np.array([[0, 1, 2, 3], [0, 2, 1, 4]], dtype=np.int32), p3, 3))
    return out
