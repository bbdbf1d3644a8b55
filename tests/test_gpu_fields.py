"""Velocity-field handles, the context's HBM budget and the error statistics
on the GPU, through the C ABI.

Fields. Algorithm 2's predictor reads the velocity field around each
particle (Sec. 2.3). A field uploaded with cs_field_upload is the input of
every CNN-SNS call that names it; two fields on one mesh must each give the
call their own predictions, while the hosts stay those of plain SNS. The
device's predictions are deterministic, so the oracle's walk given the
predictions of the same field (taken through cs_predict on the same grid
velocity) must match every start, path, status and host bit for bit; the
predictions themselves are checked against the FP64 forward pass on a sample
(6e-2 of the output scale, the BF16 bound of the other predictor tests).
"""

import numpy as np
import pytest

import oracle
from oracle import cnn, metrics
from workloads import make_case, element_node_particles
from workloads.fields import fourier_modes_2d, fourier_modes_3d
from workloads.weights import init_weights

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


def _small_fc2(dim, seed):
    flat = init_weights(dim, seed)
    o = cnn.spec(dim)
    fc2 = sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in o[:-1])
    flat[fc2:] *= 0.25
    return flat


def _oracle_pred_u(om, u_nodal):
    cen = om.pred_centres()
    return oracle.p1_interpolate(om.conn, om.v0, om.M, u_nodal, cen, om.locate(cen))


@pytest.mark.parametrize("name,kw,stride", [("tg2d", {"n_side": 101, "cfl": 8}, 3),
                                            ("abc3d", {"n_side": 15, "cfl": 8}, 3)])
def test_two_fields_give_each_call_its_own_predictions(ctx, name, kw, stride):
    import torch
    c = make_case(name, **kw)
    dim = c.dim
    flat = _small_fc2(dim, 12)
    ctx.load_predictor(dim, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=stride)
    modes = fourier_modes_2d if dim == 2 else fourier_modes_3d
    fields = [c.u, modes(c.xyz, 501)]
    handles = [ctx.upload_field(mesh, u) for u in fields]
    # particles that are not the mesh nodes: one per (element, node) pair,
    # starting from the element, with the velocity of field 0
    x, u, start = element_node_particles(c)
    xd, ud, sd = _dev(x), _dev(u), _dev(start.astype(np.int32))
    cells = int(np.prod(om.pgrid))
    preds = []
    for k, (uf, f) in enumerate(zip(fields, handles)):
        got = ctx.track(mesh, xd, ud, c.dt, start=sd, mode="cnn", field=f, start_out=True)
        # the same field through the mesh's stored grid velocity and cs_predict
        ctx.grid_velocity(mesh, _dev(uf))
        dhat = torch.empty((cells, dim), dtype=torch.float32, device="cuda")
        ctx.predict(mesh, c.dt, out=dhat)
        torch.cuda.synchronize()
        got = {kk: v.cpu().numpy() for kk, v in got.items()}
        dh = dhat.cpu().numpy()
        preds.append(dh)
        want = om.track(x, u, c.dt, start=start, mode="cnn", dhat=dh)
        st = np.where(want["path_len"] > 0, want["start"], -1)
        for kk, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                        ("status", want["status"]), ("start", st)):
            bad = np.nonzero(got[kk] != ref)[0]
            assert bad.size == 0, (k, kk, bad.size)
        plain = om.track(x, u, c.dt, start=start, mode="sns")
        assert np.array_equal(got["host"], plain["host"])
        # the predictions of this field against the FP64 forward pass
        Uref = _oracle_pred_u(om, uf)
        rng = np.random.default_rng(5 + k)
        pick = np.unique(np.concatenate([[0, cells - 1], rng.integers(0, cells, 300)]))
        w = cnn.windows(Uref.reshape(tuple(int(v) for v in om.pgrid[::-1]) + (dim,)), pick,
                        dim, c.dt / om.ps)
        ref = cnn.forward(dim, cnn.unpack(dim, flat), w)
        assert np.abs(dh[pick] - ref).max() <= 6e-2 * np.abs(ref).max(), k
    # the two fields predict differently, so the calls did not share a field
    assert np.abs(preds[0] - preds[1]).max() > 0.1 * np.abs(preds[0]).max()
    for f in handles:
        f.release()
    mesh.release()


def test_field_follows_a_predictor_grid_change(ctx):
    """A field uploaded before cs_predictor_grid is resampled to the new grid
    at its next use: its CNN-SNS call then equals the oracle's walk with the
    predictions of the nodal field on the new grid."""
    import torch
    c = make_case("tg2d", n_side=91, cfl=8)
    ctx.load_predictor(2, _small_fc2(2, 3))
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    f = ctx.upload_field(mesh, c.u)
    for stride in (3, 5):
        mesh.set_predictor_grid(stride)
        om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=stride)
        start = mesh.node_start_elements()
        got = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, start=_dev(start), mode="cnn",
                        field=f)
        ctx.grid_velocity(mesh, _dev(c.u))
        dhat = torch.empty((int(np.prod(om.pgrid)), 2), dtype=torch.float32, device="cuda")
        ctx.predict(mesh, c.dt, out=dhat)
        torch.cuda.synchronize()
        want = om.track(c.x, c.u, c.dt, start=start, mode="cnn",
                        dhat=dhat.cpu().numpy())
        for k in ("host", "path_len", "status"):
            assert np.array_equal(got[k].cpu().numpy(), want[k]), (stride, k)
    mesh.release()


def test_field_errors(ctx):
    import paper_2412_18379_gb300 as cs
    a = make_case("tg2d", n_side=41, cfl=4)
    b = make_case("tg2d", n_side=31, cfl=4)
    ctx.load_predictor(2, _small_fc2(2, 4))
    ma = ctx.upload_mesh(a.xyz, a.conn)
    mb = ctx.upload_mesh(b.xyz, b.conn)
    fb = ctx.upload_field(mb, b.u)
    start = _dev(ma.node_start_elements())
    x, u = _dev(a.x), _dev(a.u)
    # a field of another mesh
    with pytest.raises(cs.CsError) as e:
        ctx.track(ma, x, u, a.dt, mode="cnn", field=fb)
    assert e.value.code == -1
    # CNN-SNS on particles that are not the nodes needs a field
    with pytest.raises(cs.CsError) as e:
        ctx.track(ma, x, u, a.dt, start=start, mode="cnn")
    assert e.value.code == -1 and "field" in str(e.value)
    # a released field is unknown; releasing a mesh releases its fields
    fa = ctx.upload_field(ma, a.u)
    fa_id = fa.id
    fa.release()
    with pytest.raises(cs.CsError):
        ctx.track(ma, x, u, a.dt, start=start, mode="cnn", field=fa_id)
    fb_id = fb.id
    mb.release()
    with pytest.raises(cs.CsError):
        ctx._check(ctx.lib.cs_field_release(ctx.h, fb_id))
    ma.release()


def test_hbm_budget():
    """Every device allocation counts against the context's budget: a mesh
    that does not fit is refused with CS_ENOMEM and leaves nothing behind,
    and so is a serving arena larger than what is left."""
    import paper_2412_18379_gb300 as cs
    c = make_case("tg2d", n_side=101)
    probe = cs.Context(0)
    m = probe.upload_mesh(c.xyz, c.conn)
    need, budget = probe.memory_usage()
    assert budget == 0 and need >= m.info()["device_bytes"] > 0
    probe.close()
    small = cs.Context(0, hbm_budget=need // 2)
    with pytest.raises(cs.CsError) as e:
        small.upload_mesh(c.xyz, c.conn)
    assert e.value.code == -2 and "budget" in str(e.value)
    assert small.memory_usage() == (0, need // 2)
    small.close()
    roomy = cs.Context(0, hbm_budget=need + (64 << 20))
    m = roomy.upload_mesh(c.xyz, c.conn)
    used, budget = roomy.memory_usage()
    assert used <= budget
    with pytest.raises(cs.CsError) as e:
        roomy.serve_start(slots=2, arena_bytes=budget - used + (1 << 20))
    assert e.value.code == -2
    roomy.serve_start(slots=2, arena_bytes=32 << 20)
    assert roomy.memory_usage()[0] <= budget
    roomy.serve_stop()
    m.release()
    assert roomy.memory_usage()[0] < used
    roomy.close()


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 121, "cfl": 8}),
                                     ("abc3d", {"n_side": 13, "cfl": 8})])
def test_error_statistics_match_the_oracle(ctx, name, kw):
    """err (Sec. 3.1: centroid of the tracking origin to centroid of the host)
    and the displacement error |dhat s - (x_p - x)| against oracle.metrics on
    the same starts, hosts and predictions: counts exact, maxima and means to
    1e-12 relative (FP64 sums in another order)."""
    import torch
    c = make_case(name, **kw)
    dim = c.dim
    ctx.load_predictor(dim, _small_fc2(dim, 7))
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    x, u = _dev(c.x), _dev(c.u)
    cells = int(np.prod(om.pgrid))
    cent = metrics.centroids(c.xyz, c.conn)
    for mode in ("sns", "cnn"):
        out = ctx.track(mesh, x, u, c.dt, mode=mode, start_out=True)
        dhat = None
        if mode == "cnn":
            dhat = torch.empty((cells, dim), dtype=torch.float32, device="cuda")
            ctx.predict(mesh, c.dt, out=dhat)
        st = ctx.track_error(mesh, x, u, c.dt, out["host"], start=out["start"], dhat=dhat)
        torch.cuda.synchronize()
        e = metrics.err(cent, out["start"].cpu().numpy(), out["host"].cpu().numpy())
        ok = np.isfinite(e)
        assert st["n_err"] == ok.sum() > 0
        assert np.isclose(st["err_mean"], e[ok].mean(), rtol=1e-12, atol=0)
        assert np.isclose(st["err_max"], e[ok].max(), rtol=1e-12, atol=0)
        if mode == "cnn":
            xp = c.x - c.u * c.dt
            dh = dhat.cpu().numpy()
            pc = om.cnn_origin_cells(c.x, dh)[0]    # the cell the walk's start rule reads
            dd = metrics.displacement_error(dh[pc], om.ps, c.x, xp)
            assert st["n_disp"] == np.isfinite(dd).sum() == c.n_particles
            assert np.isclose(st["disp_mean"], np.nanmean(dd), rtol=1e-12, atol=0)
            assert np.isclose(st["disp_max"], np.nanmax(dd), rtol=1e-12, atol=0)
        else:
            assert st["n_disp"] == 0
    mesh.release()
