"""Pins for the oracle's point location and walk (CPU only).

Each test checks the oracle against something other than itself: the paper's
literal determinant formula, hand-derived geometry, combinatorial facts of
the mesh, closed forms, brute force, or the paper's printed tables.
"""

import os

import numpy as np
import pytest

import oracle
from oracle import metrics
from workloads import make_case, mesh_2d, mesh_3d
from workloads.meshes import tie_meshes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


# --------------------------------------------------------------------------
# barycentric coordinates (Sec. 2.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("dim", [2, 3])
def test_bary_matches_determinant_ratio(dim):
    """Inverse-affine lambda == the paper's |S_i|/|S_0| (different arithmetic)."""
    rng = np.random.default_rng(7)
    for _ in range(200):
        verts = rng.uniform(-1, 1, size=(dim + 1, dim))
        conn = np.arange(dim + 1, dtype=np.int32)[None]
        try:
            v0, M = oracle.inverse_affine(verts, conn)
        except ValueError:
            continue
        vol = abs(np.linalg.det(verts[1:] - verts[0]))
        if vol < 1e-3:
            continue
        p = rng.uniform(-2, 2, size=dim)
        lam = oracle.bary(v0[0], M[0], p)
        ref = oracle.bary_det(verts, p)
        assert np.allclose(lam, ref, rtol=0, atol=1e-9 / vol)
        # partition of unity and reproduction of the point
        assert abs(lam.sum() - 1.0) < 1e-12
        assert np.allclose(lam @ verts, p, atol=1e-10)


@pytest.mark.parametrize("dim", [2, 3])
def test_bary_special_points(dim):
    """lambda = e_i at vertex i, 1/(d+1) at the centroid."""
    xyz, conn = (mesh_2d(11)[:2] if dim == 2 else mesh_3d(5)[:2])
    v0, M = oracle.inverse_affine(xyz, conn)
    for l in range(0, conn.shape[0], max(1, conn.shape[0] // 50)):
        for i in range(dim + 1):
            lam = oracle.bary(v0[l], M[l], xyz[conn[l, i]])
            e = np.zeros(dim + 1)
            e[i] = 1.0
            assert np.allclose(lam, e, atol=1e-13)
        lam = oracle.bary(v0[l], M[l], xyz[conn[l]].mean(axis=0))
        assert np.allclose(lam, 1.0 / (dim + 1), atol=1e-13)


def test_degenerate_element_rejected():
    xyz = np.array([[0, 0], [1, 1], [2, 2.0]])
    with pytest.raises(ValueError):
        oracle.inverse_affine(xyz, np.array([[0, 1, 2]], dtype=np.int32))


# --------------------------------------------------------------------------
# neighbours m_i^l (Sec. 2.2)
# --------------------------------------------------------------------------

@pytest.mark.parametrize("which", ["2d", "3d"])
def test_neighbors_match_bruteforce(which):
    if which == "2d":
        xyz, conn, _ = mesh_2d(21)
        dim = 2
    else:
        xyz, conn, _ = mesh_3d(5)
        dim = 3
    a = oracle.neighbors(dim, conn)
    b = oracle.neighbors(dim, conn, brute=True)
    assert (a == b).all()
    # symmetry: l is a neighbour of each of its neighbours
    for l in range(conn.shape[0]):
        for m in a[l]:
            if m >= 0:
                assert l in a[m]
    # a face on the boundary has all its vertices on the square/cube boundary
    on_bnd = ((xyz == 0.0) | (xyz == 1.0)).any(axis=1)
    ls, fs = np.nonzero(a < 0)
    for l, f in zip(ls, fs):
        face = np.delete(conn[l], f)
        assert on_bnd[face].all()


def test_nonmanifold_rejected():
    conn = np.array([[0, 1, 2], [0, 1, 3], [0, 1, 4]], dtype=np.int32)
    with pytest.raises(ValueError):
        oracle.neighbors(2, conn)


# --------------------------------------------------------------------------
# result definition: lowest user id among elements containing x_p
# --------------------------------------------------------------------------

def test_two_triangles_golden():
    xyz = np.array([[0, 0], [1, 0], [1, 1], [0, 1.0]])
    conn = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    v0, M = oracle.inverse_affine(xyz, conn)
    rows = _load("two_triangles.txt")
    pts = np.array([[float(r[0]), float(r[1])] for r in rows])
    want = np.array([int(r[2]) for r in rows])
    got = oracle.locate_bruteforce(v0, M, pts)
    assert (got == want).all(), (got, want)
    # relabelling the elements moves the tie to the other triangle
    conn2 = conn[::-1].copy()
    v0, M = oracle.inverse_affine(xyz, conn2)
    got2 = oracle.locate_bruteforce(v0, M, pts)
    relabel = np.where(want >= 0, 1 - want, -1)
    relabel[2] = 0          # diagonal: both contain it, id 0 is now the upper-left one
    relabel[3] = 0
    relabel[6] = 0
    assert (got2 == relabel).all(), (got2, relabel)


def test_kuhn_cube_diagonal_tie():
    """The main diagonal is an edge of all six Kuhn tets of a cube, so its
    midpoint belongs to every one of them and id 0 wins; any point of a
    face of the cube belongs only to tets that have that face."""
    xyz, conn, _ = mesh_3d(2, 0.0, 0)
    v0, M = oracle.inverse_affine(xyz, conn)
    assert conn.shape[0] == 6
    got = oracle.locate_bruteforce(v0, M, np.array([[0.5, 0.5, 0.5]]))
    assert got[0] == 0
    # every tet contains the diagonal midpoint
    for l in range(6):
        lam = oracle.bary(v0[l], M[l], np.array([0.5, 0.5, 0.5]))
        assert lam.min() >= -1e-12


@pytest.mark.parametrize("which", ["2d", "3d"])
def test_vertex_points_lowest_incident_element(which):
    """A point at a mesh vertex lies in exactly the elements that own the
    vertex (lambda = e_i there and every other element misses it), so its
    host is the lowest incident user id -- a combinatorial fact."""
    if which == "2d":
        xyz, conn, _ = mesh_2d(31, 0.3, 5)
    else:
        xyz, conn, _ = mesh_3d(6, 0.1, 5)
    v0, M = oracle.inverse_affine(xyz, conn)
    host = oracle.locate_bruteforce(v0, M, xyz)
    lowest = np.full(xyz.shape[0], np.iinfo(np.int32).max)
    for l in range(conn.shape[0]):
        for v in conn[l]:
            lowest[v] = min(lowest[v], l)
    assert (host == lowest).all()
    assert (oracle.node_elements(xyz.shape[0], conn) == lowest).all()


def test_edge_midpoints_2d():
    """The midpoint of an interior edge lies in the two triangles that share
    it (to within rounding, absorbed by eps) and in no other."""
    xyz, conn, _ = mesh_2d(21, 0.3, 6)
    v0, M = oracle.inverse_affine(xyz, conn)
    nbr = oracle.neighbors(2, conn)
    pts, want = [], []
    for l in range(0, conn.shape[0], 3):
        for f in range(3):
            m = nbr[l, f]
            if m < 0:
                continue
            a, b = np.delete(conn[l], f)
            pts.append(0.5 * (xyz[a] + xyz[b]))
            want.append(min(l, m))
    got = oracle.locate_bruteforce(v0, M, np.array(pts))
    assert (got == np.array(want)).all()


def _orient(a, b, c):
    return (b[..., 0] - a[..., 0]) * (c[..., 1] - a[..., 1]) - \
        (b[..., 1] - a[..., 1]) * (c[..., 0] - a[..., 0])


def test_host_matches_orientation_predicate_2d():
    """On random interior points, the host agrees with a point-in-triangle
    test by orientation signs (no barycentric arithmetic)."""
    xyz, conn, _ = mesh_2d(31, 0.3, 8)
    v0, M = oracle.inverse_affine(xyz, conn)
    rng = np.random.default_rng(3)
    pts = rng.uniform(0.0, 1.0, size=(3000, 2))
    host = oracle.locate_bruteforce(v0, M, pts)
    T = xyz[conn]                                       # [n_e, 3, 2]
    for q in range(pts.shape[0]):
        p = pts[q]
        s0 = _orient(T[:, 1], T[:, 2], p)
        s1 = _orient(T[:, 2], T[:, 0], p)
        s2 = _orient(T[:, 0], T[:, 1], p)
        area = _orient(T[:, 0], T[:, 1], T[:, 2])
        inside = (s0 * area > 0) & (s1 * area > 0) & (s2 * area > 0)
        hits = np.nonzero(inside)[0]
        assert hits.size == 1 and host[q] == hits[0]


@pytest.mark.parametrize("case", [("rotation2d", {}), ("tg2d", {"n_side": 41}),
                                  ("abc3d", {"n_side": 7})])
def test_bucketed_equals_bruteforce(case):
    name, kw = case
    c = make_case(name, **kw)
    m = oracle.Mesh(c.xyz, c.conn)
    rng = np.random.default_rng(11)
    xp = oracle.departure(c.x, c.u, c.dt)
    extra = rng.uniform(-0.05, 1.05, size=(2000, c.dim))
    pts = np.concatenate([xp, c.xyz, extra, c.xyz[:50] + 1e-13, c.xyz[:50] - 1e-13])
    a = oracle.locate_bruteforce(m.v0, m.M, pts)
    for g in (3, 17):
        b = oracle.locate_bucketed(m.xyz, m.conn, m.v0, m.M, pts, g=g)
        assert (a == b).all()


# --------------------------------------------------------------------------
# Algorithm 1
# --------------------------------------------------------------------------

def _strip(n):
    """1 x n strip of unit squares, each split by the diagonal (k,0)-(k+1,1)
    into U_k = ((k,0),(k+1,1),(k,1)) and L_k = ((k,0),(k+1,0),(k+1,1))."""
    xyz = np.array([[k, 0.0] for k in range(n + 1)] + [[k, 1.0] for k in range(n + 1)])
    top = lambda k: n + 1 + k
    conn = []
    for k in range(n):
        conn.append([k, top(k + 1), top(k)])                                # U_k
        conn.append([k, k + 1, top(k + 1)])                                 # L_k
    return xyz, np.array(conn, dtype=np.int32)


def test_walk_strip_path_length():
    """Walking right from U_0 to a point of L_j: in U_k the only negative
    coordinate is the one across the diagonal (to L_k); in L_k it is the one
    across the right edge (to U_{k+1}). So the path is U_0, L_0, ..., U_j, L_j
    and I_t = 2j + 2."""
    n = 12
    xyz, conn = _strip(n)
    v0, M = oracle.inverse_affine(xyz, conn)
    nbr = oracle.neighbors(2, conn)
    for j in range(n):
        p = np.array([[j + 0.75, 0.25]])
        end, it, reason = oracle.walk(v0, M, nbr, p, np.array([0], dtype=np.int32), cap=1000)
        assert reason[0] == oracle.CONTAINED
        assert end[0] == 2 * j + 1
        assert it[0] == 2 * j + 2
    # beyond the right end the walk leaves through the boundary
    end, it, reason = oracle.walk(v0, M, nbr, np.array([[n + 0.5, 0.25]]),
                                  np.array([0], dtype=np.int32), cap=1000)
    assert reason[0] == oracle.BOUNDARY and end[0] == 2 * n - 1 and it[0] == 2 * n
    # a cap below the path length stops it after exactly `cap` evaluations
    end, it, reason = oracle.walk(v0, M, nbr, np.array([[n - 0.25, 0.25]]),
                                  np.array([0], dtype=np.int32), cap=5)
    assert reason[0] == oracle.CAP and it[0] == 5 and end[0] == 4


@pytest.mark.parametrize("case", tie_meshes(), ids=lambda c: c[0])
def test_walk_equal_minima_leave_through_lowest_local_index(case):
    """R4 (Eq. 5 leaves ties open): among exactly equal smallest coordinates
    the walk leaves through the lowest local index. In element 0 of each mesh
    p has equal negative coordinates for faces 1..d (M is the identity, so
    they are exact). Face 1 is the lowest of them. Where element 1 lies
    across face 1, the walk steps into it and stops there: I_t = 2,
    FOUND. Where it lies across a higher face, face 1 is a boundary face,
    so the walk ends there after one evaluation and the exact search finds
    element 1 (FOUND_VIA_FALLBACK). Picking the last equal minimum instead,
    or scanning the faces in reverse, swaps the two outcomes."""
    name, xyz, conn, p, face = case
    m = oracle.Mesh(xyz, conn)
    lam = oracle.bary(m.v0[0], m.M[0], p[0])
    assert np.all(lam[1:] == lam[1]) and lam[1] < 0
    assert m.nbr[0][face] == 1 and (m.nbr[0] >= 0).sum() == 1
    end, it, reason = oracle.walk(m.v0, m.M, m.nbr, p, np.array([0], dtype=np.int32))
    r = m.track(p, np.zeros_like(p), 0.0, start=np.array([0], dtype=np.int32))
    assert r["host"][0] == 1
    if face == 1:
        assert reason[0] == oracle.CONTAINED and end[0] == 1 and it[0] == 2
        assert r["status"][0] == oracle.ST_FOUND and r["path_len"][0] == 2
    else:
        assert reason[0] == oracle.BOUNDARY and end[0] == 0 and it[0] == 1
        assert r["status"][0] == oracle.ST_FALLBACK and r["path_len"][0] == 1


def test_walk_start_inside_is_one_step():
    c = make_case("rotation2d")
    m = oracle.Mesh(c.xyz, c.conn)
    # dt = 0: every particle sits on its node, inside its start element
    r = m.track(c.x, c.u, 0.0)
    assert (r["path_len"] == 1).all()
    assert (r["status"] == oracle.ST_FOUND).all()
    assert (r["host"] == m.node_elem).all()


@pytest.mark.parametrize("case", [("rotation2d", {}), ("tg2d", {"n_side": 61, "cfl": 8}),
                                  ("abc3d", {"n_side": 9, "cfl": 6})])
def test_track_invariants(case):
    name, kw = case
    c = make_case(name, **kw)
    m = oracle.Mesh(c.xyz, c.conn)
    r = m.track(c.x, c.u, c.dt)
    host, st = r["host"], r["status"]
    found = host >= 0
    # every located point has all barycentric coordinates >= -1e-12
    for q in np.nonzero(found)[0][::7]:
        assert oracle.bary(m.v0[host[q]], m.M[host[q]], r["xp"][q]).min() >= -1e-12
    # a walk that ended by containment ended in an element that contains x_p,
    # and the canonical host is the lowest such id
    cont = r["reason"] == oracle.CONTAINED
    assert (host[cont] <= r["end"][cont]).all()
    assert (st[cont] == oracle.ST_FOUND).all()
    assert ((st == oracle.ST_OUTSIDE) == (host < 0)).all()
    # host does not depend on the start element
    rng = np.random.default_rng(5)
    st2 = rng.integers(0, m.n_e, size=c.n_particles).astype(np.int32)
    r2 = m.track(c.x, c.u, c.dt, start=st2)
    assert (r2["host"] == host).all()
    # nor on the start rule
    r3 = m.track(c.x, c.u, c.dt, mode="asg")
    assert (r3["host"] == host).all()
    assert r3["path_len"].mean() <= r["path_len"].mean()


def test_rotation_closed_form_departure():
    """Solid-body rotation: the exact foot is c + R(-dt)(x - c); the first-
    order foot x - u dt differs from it by at most |x - c| dt^2 / 2 (the
    Taylor remainder of the rotation), and both feet are located."""
    c = make_case("rotation2d")
    xp = oracle.departure(c.x, c.u, c.dt)
    assert np.array_equal(xp, c.x - c.u * c.dt)
    ctr = np.array([0.5, 0.5])
    ang = -c.dt
    R = np.array([[np.cos(ang), -np.sin(ang)], [np.sin(ang), np.cos(ang)]])
    exact = ctr + (c.x - ctr) @ R.T
    r = np.linalg.norm(c.x - ctr, axis=1)
    assert (np.linalg.norm(xp - exact, axis=1) <= 0.5 * r * c.dt ** 2 * (1 + 1e-9) + 1e-15).all()
    m = oracle.Mesh(c.xyz, c.conn)
    h_exact = m.locate(exact)
    # the exact foot of a rotation stays inside the disc of radius |x - c|;
    # corners of the square have |x - c| > 0.5, so only they may leave
    inside_sq = ((exact >= 0) & (exact <= 1)).all(axis=1)
    assert ((h_exact >= 0) == inside_sq).all()


def test_seed_grid_contains_centres():
    c = make_case("tg2d", n_side=41)
    m = oracle.Mesh(c.xyz, c.conn, grid=23)
    cen = oracle.grid_centres(m.lo, m.hi, m.grid)
    assert (m.seed >= 0).all()
    for q in range(0, cen.shape[0], 5):
        lam = oracle.bary(m.v0[m.seed[q]], m.M[m.seed[q]], cen[q])
        assert lam.min() >= -1e-12
    # every centre lies in its own cell
    assert (m.cells(cen) == np.arange(cen.shape[0])).all()


def test_p1_interpolation_exact_for_linear_fields():
    c = make_case("abc3d", n_side=6)
    m = oracle.Mesh(c.xyz, c.conn, grid=7)
    A = np.array([[0.3, -1.0, 2.0], [1.5, 0.2, -0.7], [-0.4, 0.9, 0.1]])
    b = np.array([0.1, -0.2, 0.3])
    u_nodal = c.xyz @ A.T + b
    cen = oracle.grid_centres(m.lo, m.hi, m.grid)
    u = oracle.p1_interpolate(m.conn, m.v0, m.M, u_nodal, cen, m.seed)
    assert np.allclose(u, cen @ A.T + b, atol=1e-12)


# --------------------------------------------------------------------------
# reported metrics (Sec. 3)
# --------------------------------------------------------------------------

def test_opt_reproduces_paper_tables():
    for t, metric, sns, cnn, printed in _load("opt_tables.txt"):
        got = 100.0 * metrics.opt(float(sns), float(cnn))
        assert abs(got - float(printed)) <= 0.0015, (t, metric, sns, cnn, printed, got)


def test_err_is_centroid_distance():
    xyz = np.array([[0, 0], [1, 0], [1, 1], [0, 1.0]])
    conn = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    cent = metrics.centroids(xyz, conn)
    assert np.allclose(cent, [[2 / 3, 1 / 3], [1 / 3, 2 / 3]])
    e = metrics.err(cent, np.array([0, 1, 0, -1]), np.array([1, 1, 0, 0]))
    assert np.allclose(e[:3], [np.sqrt(2) / 3, 0, 0]) and np.isnan(e[3])


def test_displacement_error_closed_forms():
    """A prediction equal to the true displacement (exact in float32 here:
    dyadic values) has error 0; one off by (3, 4) cells of size (0.5, 0.25)
    has error |(1.5, 1.0)| = sqrt(3.25); a non-finite departure point gives NaN."""
    x = np.array([[0.25, 0.5], [0.0, 0.0], [1.0, 1.0]])
    xp = np.array([[0.75, 0.0], [0.5, -0.5], [np.inf, 1.0]])
    s = np.array([0.5, 0.25])
    exact = (xp - x) / s
    exact[2] = 0.0
    e = metrics.displacement_error(exact.astype(np.float32), s, x, xp)
    assert e[0] == 0.0 and e[1] == 0.0 and np.isnan(e[2])
    off = exact + np.array([3.0, 4.0])
    e = metrics.displacement_error(off.astype(np.float32), s, x, xp)
    assert np.isclose(e[0], np.sqrt(3.25), rtol=0, atol=1e-15)


def test_oracle_threads_do_not_change_results():
    """The all-core CPU baseline runs the oracle's particle loops on OpenMP
    threads; particles are independent, so every output is the same bits as
    the single-threaded run."""
    c = make_case("tg2d", n_side=151, cfl=8)
    m = oracle.Mesh(c.xyz, c.conn, brute_limit=0)
    oracle.set_threads(1)
    one = m.track(c.x, c.u, c.dt)
    try:
        used = oracle.set_threads(4)
        many = m.track(c.x, c.u, c.dt)
    finally:
        oracle.set_threads(1)
    assert used in (1, 4)
    for k in ("host", "path_len", "status", "start"):
        assert np.array_equal(one[k], many[k]), k
