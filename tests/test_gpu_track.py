"""Parity of the CUDA particle-location path against the CPU oracle.

Every GPU call goes through the C ABI (libcnnsns.so via the ctypes binding).
Bar: bit-exact host ids, path lengths, statuses and start elements.
"""

import numpy as np
import pytest

import oracle
from workloads import make_case

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2412_18379_gb300 as cs
    from paper_2412_18379_gb300 import build
    build.build()
    c = cs.Context(0)
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(ctx, mesh, case, mode="sns", start=None, dt=None, u=None):
    import torch
    x = _dev(case.x)
    uu = _dev(case.u if u is None else u)
    st = None if start is None else _dev(start.astype(np.int32))
    out = ctx.track(mesh, x, uu, case.dt if dt is None else dt, start=st, mode=mode,
                    start_out=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(got, want, name=""):
    for k in ("host", "path_len", "status", "start"):
        a, b = got[k], want[k]
        bad = np.nonzero(a != b)[0]
        assert bad.size == 0, "%s %s differs at %d particles, first %s: gpu %s oracle %s" % (
            name, k, bad.size, bad[:5], a[bad[:5]], b[bad[:5]])


def _oracle_out(om, r):
    # the oracle reports starts in user ids; -1 where no walk ran
    start = np.where(r["path_len"] > 0, r["start"], -1)
    return dict(host=r["host"], path_len=r["path_len"], status=r["status"], start=start)


CASES = [
    ("rotation2d", {}),
    ("tg2d", {"n_side": 201, "cfl": 1}),
    ("tg2d", {"n_side": 201, "cfl": 16}),
    ("abc3d", {"n_side": 21, "cfl": 4}),
    ("abc3d", {"n_side": 21, "cfl": 20}),
    ("hole2d", {"n_side": 61}),      # non-convex: walks blocked by the hole
    ("hole2d", {"n_side": 121}),
    ("sphere3d", {"n_side": 25}),    # non-convex in 3-D: walks blocked by the ball
    ("sphere3d", {"n_side": 41}),
]


@pytest.mark.parametrize("name,kw", CASES)
@pytest.mark.parametrize("mode", ["sns", "asg"])
def test_track_parity(ctx, name, kw, mode):
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    got = _run(ctx, mesh, c, mode=mode)
    want = _oracle_out(om, om.track(c.x, c.u, c.dt, mode=mode))
    _compare(got, want, "%s %s %s" % (name, kw, mode))
    mesh.release()


def test_non_convex_domain_uses_the_exact_search(ctx):
    """Walks that meet the hole's boundary with the departure point beyond it
    end in the exact search (FOUND_VIA_FALLBACK); departure points in the hole
    or outside the square are OUTSIDE. Same bits as the oracle."""
    c = make_case("hole2d", n_side=61)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    got = _run(ctx, mesh, c)
    _compare(got, _oracle_out(om, om.track(c.x, c.u, c.dt)), "hole2d")
    counts = np.bincount(got["status"], minlength=4)
    assert counts[2] > 20 and counts[1] > 100, counts
    r = np.linalg.norm(c.x - c.u * c.dt - 0.5, axis=1)
    assert (got["host"][r < 0.09] == -1).all()            # inside the hole
    mesh.release()


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 101, "cfl": 8}),
                                     ("abc3d", {"n_side": 13, "cfl": 8})])
def test_random_starts(ctx, name, kw):
    """Explicit user-id starts, including -1 (walk skipped)."""
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    rng = np.random.default_rng(21)
    start = rng.integers(0, c.n_elements, size=c.n_particles).astype(np.int32)
    start[::97] = -1
    got = _run(ctx, mesh, c, start=start)
    want = _oracle_out(om, om.track(c.x, c.u, c.dt, start=start))
    _compare(got, want)


def test_mesh_tables(ctx):
    c = make_case("tg2d", n_side=51)
    mesh = ctx.upload_mesh(c.xyz, c.conn, asg_grid=37)
    om = oracle.Mesh(c.xyz, c.conn, grid=37)
    assert (mesh.node_start_elements() == om.node_elem).all()
    assert (mesh.seed_grid() == om.seed).all()
    inf = mesh.info()
    assert inf["asg_grid"] == [37, 37] and inf["record_bytes"] == 48
    assert inf["step_cap"] == om.cap


def test_edge_cases(ctx):
    import torch
    c = make_case("rotation2d")
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    # dt = 0: every particle is inside its start element
    got = _run(ctx, mesh, c, dt=0.0)
    assert (got["path_len"] == 1).all() and (got["status"] == 0).all()
    assert (got["host"] == om.node_elem).all()
    # non-finite velocities -> INVALID, the rest unaffected
    u = c.u.copy()
    u[::13, 0] = np.nan
    u[5, 1] = np.inf
    got = _run(ctx, mesh, c, u=u)
    want = _oracle_out(om, om.track(c.x, u, c.dt))
    _compare(got, want)
    assert (got["status"][::13] == 3).all()
    # large dt throws many particles out of the square
    got = _run(ctx, mesh, c, dt=c.dt * 8)
    want = _oracle_out(om, om.track(c.x, c.u, c.dt * 8))
    _compare(got, want)
    assert (got["status"] == 1).sum() > 100
    # n = 0 is a no-op
    e = torch.empty((0, 2), dtype=torch.float64, device="cuda")
    s = torch.empty(0, dtype=torch.int32, device="cuda")
    out = ctx.track(mesh, e, e, 0.1, start=s)
    assert out["host"].numel() == 0


def test_points_on_vertices_and_edges(ctx):
    """Points exactly at vertices and on edges: the lowest id must win."""
    c = make_case("tg2d", n_side=41)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    nbr = om.nbr
    pts = [c.xyz]
    mids = []
    for l in range(0, c.n_elements, 2):
        for f in range(3):
            a, b = np.delete(c.conn[l], f)
            mids.append(0.5 * (c.xyz[a] + c.xyz[b]))
    pts = np.concatenate([c.xyz, np.array(mids)])
    zeros = np.zeros_like(pts)
    rng = np.random.default_rng(3)
    start = rng.integers(0, c.n_elements, size=pts.shape[0]).astype(np.int32)
    import torch
    out = ctx.track(mesh, _dev(pts), _dev(zeros), 0.0, start=_dev(start), start_out=True)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    want = _oracle_out(om, om.track(pts, zeros, 0.0, start=start))
    _compare(got, want)
    del nbr


def test_host_path_matches_device_path(ctx):
    c = make_case("abc3d", n_side=11, cfl=10)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    dev = _run(ctx, mesh, c, mode="asg")
    host = ctx.track_host(mesh, c.x, c.u, c.dt, mode="asg", start_out=True)
    for k in ("host", "path_len", "status", "start"):
        assert (dev[k] == host[k]).all()


def test_stats_and_determinism(ctx):
    import torch
    c = make_case("tg2d", n_side=151, cfl=12)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    x, u = _dev(c.x), _dev(c.u)
    a = ctx.track(mesh, x, u, c.dt)
    b = ctx.track(mesh, x, u, c.dt)
    torch.cuda.synchronize()
    for k in a:
        assert torch.equal(a[k], b[k])
    s = ctx.stats(a["path_len"], a["status"])
    p = a["path_len"].cpu().numpy()
    st = a["status"].cpu().numpy()
    assert s["sum"] == p.sum() and s["max"] == p.max()
    assert [s["found"], s["outside"], s["fallback"], s["invalid"]] == \
        [int((st == k).sum()) for k in range(4)]


def test_bad_meshes_rejected(ctx):
    import paper_2412_18379_gb300 as cs
    xyz = np.array([[0, 0], [1, 0], [1, 1], [0, 1.0], [2, 2.0]])
    with pytest.raises(cs.CsError) as e:
        ctx.upload_mesh(xyz, np.array([[0, 1, 2], [0, 2, 9]]))
    assert e.value.code == -6
    with pytest.raises(cs.CsError) as e:        # degenerate (collinear)
        ctx.upload_mesh(xyz, np.array([[0, 2, 4], [0, 1, 2]]))
    assert e.value.code == -6
    with pytest.raises(cs.CsError) as e:        # an edge shared by three triangles
        ctx.upload_mesh(xyz, np.array([[0, 2, 1], [0, 2, 3], [0, 2, 4]]))
    assert e.value.code == -6


def test_full_size_tg2d_parity(ctx):
    """The 1001 x 1001 Taylor-Green workload at CFL 8, every particle."""
    c = make_case("tg2d", cfl=8)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    for mode in ("sns", "asg"):
        got = _run(ctx, mesh, c, mode=mode)
        want = _oracle_out(om, om.track(c.x, c.u, c.dt, mode=mode))
        _compare(got, want, "full tg2d " + mode)
    mesh.release()


def test_full_size_abc3d_parity(ctx):
    """The 101^3 Kuhn cube (6.0M tetrahedra) with ABC flow at CFL 8, every
    particle, plain SNS."""
    c = make_case("abc3d", cfl=8)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    got = _run(ctx, mesh, c, mode="sns")
    want = _oracle_out(om, om.track(c.x, c.u, c.dt, mode="sns"))
    _compare(got, want, "full abc3d sns")
    mesh.release()


def test_equal_minima_leave_through_the_lowest_local_index(ctx):
    """R4 on meshes whose start element has exactly equal smallest
    coordinates (Eq. 5's ties): the device takes the same exit as the oracle,
    so paths, statuses, starts and hosts match bit for bit."""
    import torch
    from workloads.meshes import tie_meshes
    for name, xyz, conn, p, face in tie_meshes():
        mesh = ctx.upload_mesh(xyz, conn)
        om = oracle.Mesh(xyz, conn, grid=mesh.info()["asg_grid"])
        pts = np.repeat(p, 64, axis=0)
        zeros = np.zeros_like(pts)
        start = np.zeros(pts.shape[0], dtype=np.int32)
        out = ctx.track(mesh, _dev(pts), _dev(zeros), 0.0, start=_dev(start), start_out=True)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        want = _oracle_out(om, om.track(pts, zeros, 0.0, start=start))
        _compare(got, want, name)
        assert (got["path_len"] == (2 if face == 1 else 1)).all(), name
        mesh.release()


def test_non_convex_3d_domain_uses_the_exact_search(ctx):
    """The cube with a ball taken out: walks that meet the ball's surface with
    the departure point beyond it end in the exact search (FOUND_VIA_FALLBACK),
    bit for bit with the oracle, and are a visible share of the particles."""
    c = make_case("sphere3d", n_side=41)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    got = _run(ctx, mesh, c)
    _compare(got, _oracle_out(om, om.track(c.x, c.u, c.dt)), "sphere3d")
    assert (got["status"] == 2).sum() > 100
    mesh.release()


@pytest.mark.parametrize("mode", ["sns", "asg", "cnn"])
def test_host_entry_point_matches_the_device_one(ctx, mode):
    """cs_track_host (copies through a device staging buffer) on page-locked
    and on pageable host arrays: results equal the device entry point's bit
    for bit, for the mesh nodes and for explicit starts with a resident
    field."""
    import torch
    from workloads.weights import init_weights
    from workloads import element_node_particles
    c = make_case("tg2d", n_side=401, cfl=8)
    ctx.load_predictor(2, init_weights(2, 12))
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    want = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode=mode, start_out=True)
    torch.cuda.synchronize()
    want = {k: v.cpu().numpy() for k, v in want.items()}
    n = c.n_particles
    pinned = dict(host=torch.full((n,), -7, dtype=torch.int32).pin_memory(),
                  path_len=torch.full((n,), -7, dtype=torch.int32).pin_memory(),
                  status=torch.full((n,), 9, dtype=torch.uint8).pin_memory(),
                  start=torch.full((n,), -7, dtype=torch.int32).pin_memory())
    for xs, us, out in ((torch.from_numpy(c.x).pin_memory(), torch.from_numpy(c.u).pin_memory(),
                         pinned), (c.x, c.u, None)):
        got = ctx.track_host(mesh, xs, us, c.dt, mode=mode, start_out=True, out=out)
        for k in ("host", "path_len", "status", "start"):
            g = got[k].numpy() if hasattr(got[k], "numpy") else got[k]
            assert np.array_equal(g, want[k]), (mode, out is None, k)
    # explicit starts (element-node particles) with a resident field
    x, u, start = element_node_particles(c)
    f = ctx.upload_field(mesh, c.u)
    want = ctx.track(mesh, _dev(x), _dev(u), c.dt, start=_dev(start), mode=mode, field=f)
    torch.cuda.synchronize()
    got = ctx.track_host(mesh, x, u, c.dt, start=start, mode=mode, field=f)
    for k in ("host", "path_len", "status"):
        assert np.array_equal(got[k], want[k].cpu().numpy()), (mode, "pairs", k)
    mesh.release()


@pytest.mark.parametrize("mode", ["sns", "asg", "cnn"])
def test_nodes_entry_point_matches_the_host_one(ctx, mode):
    """cs_track_nodes_host (the particles at the mesh's own vertex
    coordinates, only u copied in) gives the bits of cs_track_host on x = the
    vertices: in 2-D on a mesh large enough for the chunked pipeline, and in
    3-D; with the call's own u (page-locked and pageable) and with a resident
    field."""
    import torch
    from workloads.weights import init_weights
    for name, kw, stride in (("tg2d", {"n_side": 1001}, 5), ("abc3d", {"n_side": 41}, 3)):
        c = make_case(name, cfl=8, **kw)
        assert np.array_equal(c.x, c.xyz)
        ctx.load_predictor(c.dim, init_weights(c.dim, 12))
        mesh = ctx.upload_mesh(c.xyz, c.conn)
        mesh.set_predictor_grid(stride)
        want = ctx.track_host(mesh, c.x, c.u, c.dt, mode=mode, start_out=True)
        for u in (torch.from_numpy(c.u).pin_memory(), c.u):
            got = ctx.track_nodes_host(mesh, u, c.dt, mode=mode, start_out=True)
            for k in ("host", "path_len", "status", "start"):
                assert np.array_equal(got[k], want[k]), (name, mode, k)
        f = ctx.upload_field(mesh, c.u)
        want = ctx.track_host(mesh, c.x, c.u, c.dt, mode=mode, field=f)
        got = ctx.track_nodes_host(mesh, c.u, c.dt, mode=mode, field=f)
        for k in ("host", "path_len", "status"):
            assert np.array_equal(got[k], want[k]), (name, mode, "field", k)
        f.release()
        mesh.release()


@pytest.mark.parametrize("mode", ["sns", "asg", "cnn"])
def test_shards_of_one_batch_concatenate_to_the_whole(ctx, mode):
    """The multi-GPU split of one batch (bench.py --shard): each of 3 shards
    (shard_range slices, the node particles with their node's element as an
    explicit start, CNN-SNS predicting from a resident field) is located by a
    call of its own, one after the other on this GPU; concatenated, the
    results equal the whole batch's bit for bit. Every shard runs alone: no
    call waits on another."""
    import torch
    from workloads.weights import init_weights
    from paper_2412_18379_gb300.shard import shard_range
    c = make_case("tg2d", n_side=301, cfl=8)
    ctx.load_predictor(2, init_weights(2, 31))
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    f = ctx.upload_field(mesh, c.u)
    starts = mesh.node_start_elements()
    whole = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, start=_dev(starts), mode=mode, field=f,
                      start_out=True)
    torch.cuda.synchronize()
    parts = []
    for r in range(3):
        lo, hi = shard_range(c.n_particles, r, 3)
        o = ctx.track(mesh, _dev(c.x[lo:hi]), _dev(c.u[lo:hi]), c.dt, start=_dev(starts[lo:hi]),
                      mode=mode, field=f, start_out=True)
        torch.cuda.synchronize()
        parts.append({k: v.cpu().numpy() for k, v in o.items()})
    for k in ("host", "path_len", "status", "start"):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), whole[k].cpu().numpy()), k
