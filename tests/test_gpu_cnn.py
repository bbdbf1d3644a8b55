"""The learned start predictor on the GPU against the FP64 oracle.

Tolerances. The predictor computes with BF16 operands (8 significant bits,
relative rounding 2^-9) and FP32 accumulation. Each of the six layers rounds
its inputs and weights once, so the output carries a relative error of order
6 * 2 * 2^-9 ~ 2.3e-2 of its scale; tests allow 4e-2 of the output's largest
magnitude. The grid velocity is evaluated in FP32: the cell-centre offsets
carry ~1e-7 absolute error, the barycentric coordinates ~1e-7 / h relative,
so 5e-4 of the largest velocity covers h >= 1e-3 with margin. Windows are
one FP32 product: 1e-6 relative. Start elements of CNN-SNS depend on the
BF16 prediction and may differ from the FP64 oracle's where the predicted
point lies within the prediction error of an ASG cell boundary; hosts never do.
"""

import numpy as np
import pytest

import oracle
from oracle import cnn
from workloads import make_case
from workloads.weights import init_weights
from workloads.fields import fourier_modes_2d, dt_for_cfl

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


def _oracle_grid_u(om, u_nodal):
    cen = oracle.grid_centres(om.lo, om.hi, om.grid)
    return oracle.p1_interpolate(om.conn, om.v0, om.M, u_nodal, cen, om.seed)


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 101}), ("abc3d", {"n_side": 13})])
def test_grid_velocity_matches_oracle(ctx, name, kw):
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    U = torch.empty((int(np.prod(g)), c.dim), dtype=torch.float32, device="cuda")
    ctx.grid_velocity(mesh, _dev(c.u), out=U)
    torch.cuda.synchronize()
    ref = _oracle_grid_u(om, c.u)
    err = np.abs(U.cpu().numpy() - ref).max()
    assert err <= 5e-4 * np.abs(c.u).max(), err


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 61}), ("abc3d", {"n_side": 11})])
def test_windows_match_oracle(ctx, name, kw):
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    Uref = _oracle_grid_u(om, c.u)
    rng = np.random.default_rng(4)
    cells = rng.integers(0, Uref.shape[0], size=300).astype(np.int64)
    cells[:4] = [0, Uref.shape[0] - 1, g[0] - 1, g[0]]      # corners and edges
    w = ctx.windows(mesh, c.dt, cells=_dev(cells), grid=_dev(Uref.astype(np.float32)))
    torch.cuda.synchronize()
    scale = c.dt / ((om.hi - om.lo) / om.grid)
    ref = cnn.windows(Uref.astype(np.float32).reshape(tuple(g[::-1]) + (c.dim,)), cells, c.dim,
                      scale)
    assert np.allclose(w.cpu().numpy(), ref, rtol=1e-6, atol=1e-7 * np.abs(ref).max())


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("bf16", [False, True])
def test_forward_and_gradient_match_oracle(ctx, dim, bf16):
    """FP32 operands: forward and every layer's gradient within 1e-4 of the
    FP64 oracle (FP32 accumulation over at most 4096 terms). BF16 operands
    (the training arithmetic): forward within 4e-2 of the output scale; the
    gradient of layer l passes through 2 * (L - l) BF16-rounded GEMM operands
    and through the ReLU gates of a forward pass that is itself off by ~1e-2,
    so the deepest layer is allowed 1.5e-1 relative error, others 5e-2."""
    rng = np.random.default_rng(10 + dim)
    flat = init_weights(dim, 7).astype(np.float64)
    flat += 0.02 * rng.standard_normal(flat.size)
    flat = flat.astype(np.float32)
    ctx.predictor_precision(bf16)
    try:
        ctx.load_predictor(dim, flat)
        S = cnn.patch_size(dim)
        B = 96
        win = rng.standard_normal((B, dim) + (S,) * dim).astype(np.float32)
        tgt = rng.standard_normal((B, dim)).astype(np.float32)
        params = cnn.unpack(dim, flat)
        ref, acts = cnn.forward(dim, params, win.astype(np.float64), keep=True)
        out = ctx.predictor_forward(dim, _dev(win)).cpu().numpy()
        ftol = 4e-2 if bf16 else 1e-5
        assert np.abs(out - ref).max() <= ftol * np.abs(ref).max()
        # gradients of the MSE against the FP64 backward, layer by layer
        gref = cnn.pack(cnn.backward(dim, params, acts, ref, tgt.astype(np.float64)))
        g, loss = ctx.predictor_grad(dim, _dev(win), _dev(tgt))
        g = g.cpu().numpy().astype(np.float64)
        assert abs(loss - cnn.mse(ref, tgt)) <= ftol * cnn.mse(ref, tgt)
        o = 0
        for li, (_, ws, bs) in enumerate(cnn.spec(dim)):
            n = int(np.prod(ws)) + int(np.prod(bs))
            a, b = g[o:o + n], gref[o:o + n]
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            tol = (1.5e-1 if li == 0 else 5e-2) if bf16 else 1e-4
            assert rel <= tol, (ws, rel)
            o += n
    finally:
        ctx.predictor_precision(True)


@pytest.mark.parametrize("dim", [2, 3])
def test_adam_step_on_device(ctx, dim):
    """One training step over the whole batch: the update is Adam's first
    step -lr g/(|g| + eps) of the device's own gradient on the same pairs."""
    rng = np.random.default_rng(20 + dim)
    flat = init_weights(dim, 8)
    ctx.load_predictor(dim, flat)
    S = cnn.patch_size(dim)
    B = 64
    win = _dev(rng.standard_normal((B, dim) + (S,) * dim).astype(np.float32))
    tgt = _dev(rng.standard_normal((B, dim)).astype(np.float32))
    g, _ = ctx.predictor_grad(dim, win, tgt)
    g = g.cpu().numpy().astype(np.float64)
    losses = ctx.train(dim, win, tgt, batch=B, steps=1, lr=1e-3, seed=3)
    w1 = ctx.save_predictor(dim).astype(np.float64)
    want = flat.astype(np.float64) - 1e-3 * g / (np.abs(g) + 1e-8)
    big = np.abs(g) > 1e-6
    assert np.allclose(w1[big], want[big], rtol=0, atol=2e-6)
    assert np.all(np.abs(w1[~big] - flat[~big]) <= 1e-3 + 1e-6)
    assert losses.shape == (1,) and np.isfinite(losses[0])


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 121, "cfl": 8}),
                                     ("abc3d", {"n_side": 15, "cfl": 8})])
def test_track_with_given_displacements(ctx, name, kw):
    """Algorithm 2's start rule with a displacement grid drawn from a seeded
    generator: starts, paths, hosts and statuses bit for bit."""
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    rng = np.random.default_rng(6)
    dhat = rng.uniform(-12, 12, size=(int(np.prod(g)), c.dim)).astype(np.float32)
    out = ctx.track_dhat(mesh, _dev(c.x), _dev(c.u), c.dt, dhat=_dev(dhat), start_out=True)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat)
    start = np.where(want["path_len"] > 0, want["start"], -1)
    for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                   ("status", want["status"]), ("start", start)):
        assert np.array_equal(got[k], ref), k


def test_track_with_special_displacements(ctx):
    """The CNN start with displacements that are not ordinary numbers: signed
    zeros, float subnormals, values near the float range, infinities and NaN
    (a diverged predictor). x + dhat * s then lies on x, next to it, far
    outside the box (clamped to the boundary cells) or is NaN (cell 0); the
    walk from there must still end in the exact host. Starts, paths, hosts and
    statuses bit for bit."""
    import torch
    c = make_case("tg2d", n_side=61, cfl=8)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    rng = np.random.default_rng(8)
    dhat = rng.uniform(-4, 4, size=(int(np.prod(g)), c.dim)).astype(np.float32)
    special = np.array([0.0, -0.0, 1e-40, -1.4e-45, 5.9e-39, -1.17e-38, 3.0e38, -3.3e38,
                        np.inf, -np.inf, np.nan, 1.0, -0.5], dtype=np.float32)
    pick = rng.integers(0, special.size, size=dhat.shape)
    mask = rng.random(dhat.shape) < 0.5
    dhat[mask] = special[pick[mask]]
    out = ctx.track_dhat(mesh, _dev(c.x), _dev(c.u), c.dt, dhat=_dev(dhat), start_out=True)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    with np.errstate(invalid="ignore", over="ignore"):
        want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat)
    start = np.where(want["path_len"] > 0, want["start"], -1)
    for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                   ("status", want["status"]), ("start", start)):
        assert np.array_equal(got[k], ref), k
    mesh.release()


@pytest.mark.parametrize("name,kw,stride", [("tg2d", {"n_side": 121}, 3),
                                            ("abc3d", {"n_side": 13}, 1)])
def test_cnn_start_cells_next_to_cell_faces(ctx, name, kw, stride):
    """The start point y = x + dhat * s of Algorithm 2 placed on ASG cell
    faces and within 1 ulp .. 1e-9 of them, on both sides: the start element
    (the seed of y's ASG cell, whose index the device takes through its FP32
    cell filter with an FP64 fallback) and the whole walk agree with the FP64
    oracle bit for bit."""
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=stride)
    rng = np.random.default_rng(23)
    s = (om.hi - om.lo) / om.grid
    n_cell = int(np.prod(om.pgrid))
    for dh in (1.37, -2.9, 0.001):
        dhat = np.full((n_cell, c.dim), dh, dtype=np.float32)
        disp = np.float32(dh).astype(np.float64) * om.ps
        # target points on random ASG faces on every axis, then nudged
        n = 3000
        face = om.lo + rng.integers(1, om.grid, size=(n, c.dim)) * s
        nudge = np.array([0.0, 1e-16, -1e-16, 1e-13, -1e-13, 1e-11, -1e-11, 1e-9, -1e-9])
        y = face + nudge[rng.integers(0, nudge.size, size=(n, c.dim))] * np.maximum(1, np.abs(face))
        y = np.where(rng.random((n, c.dim)) < 0.2, np.nextafter(face, face + 1), y)
        x = y - disp
        keep = np.all((x > om.lo) & (x < om.hi), axis=1)
        x = np.ascontiguousarray(x[keep])
        u = np.zeros_like(x)
        start = rng.integers(0, c.n_elements, size=x.shape[0]).astype(np.int32)
        out = ctx.track_dhat(mesh, _dev(x), _dev(u), c.dt, dhat=_dev(dhat), start=_dev(start),
                             start_out=True)
        torch.cuda.synchronize()
        got = {k: v.cpu().numpy() for k, v in out.items()}
        want = om.track(x, u, c.dt, start=start, mode="cnn", dhat=dhat)
        st = np.where(want["path_len"] > 0, want["start"], -1)
        for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                       ("status", want["status"]), ("start", st)):
            assert np.array_equal(got[k], ref), (dh, k, np.nonzero(got[k] != ref)[0][:5])
        assert x.shape[0] > 500
    mesh.release()


def _oracle_cnn_dhat(om, case, flat):
    """Oracle of the predictor stage: FP64 grid velocity, the window of every
    ASG cell, FP64 forward (the prediction grid)."""
    U = _oracle_grid_u(om, case.u)
    cells = np.arange(int(np.prod(om.grid)))
    scale = case.dt / ((om.hi - om.lo) / om.grid)
    G = tuple(int(v) for v in om.grid[::-1])
    win = cnn.windows(U.reshape(G + (case.dim,)), cells, case.dim, scale)
    return cnn.forward(case.dim, cnn.unpack(case.dim, flat), win)


def test_cnn_sns_matches_oracle(ctx):
    import torch
    c = make_case("tg2d", n_side=81, cfl=8)
    flat = init_weights(2, 12)
    o = cnn.spec(2)
    fc2 = sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in o[:-1])
    flat[fc2:] *= 0.25          # predictions of a few cells, like a trained net
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    out = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode="cnn", start_out=True)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    dgrid = _oracle_cnn_dhat(om, c, flat)
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dgrid)
    dref = dgrid[om.cnn_origin_cells(c.x, dgrid)[0]]
    plain = om.track(c.x, c.u, c.dt, mode="sns")
    assert np.array_equal(got["host"], want["host"])
    assert np.array_equal(got["host"], plain["host"])          # SNS == CNN-SNS hosts
    assert np.array_equal(got["status"] == 1, want["status"] == 1)
    # where the oracle's predicted point is farther from every ASG cell
    # boundary than the BF16 error bound, the start element must agree
    s = (om.hi - om.lo) / om.grid
    frac = (c.x - om.lo) / s + dref
    dist = np.abs(frac - np.round(frac)).min(axis=1)
    safe = dist > 4e-2 * np.abs(dref).max()
    assert safe.mean() > 0.5
    assert np.array_equal(got["start"][safe], want["start"][safe])
    same = got["start"] == want["start"]
    assert np.array_equal(got["path_len"][same], want["path_len"][same])


def test_training_gains_over_plain_sns(ctx):
    """Pairs from plain SNS on random 8-mode fields, a short training run on
    the GPU, then on a held-out field CNN-SNS must walk shorter paths than
    plain SNS at CFL 8 while returning the same hosts."""
    import torch
    c = make_case("modes2d", n_side=101, cfl=8)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    ctx.load_predictor(2, init_weights(2, 0))
    rng = np.random.default_rng(42)
    x = _dev(c.x)
    wins, tgts = [], []
    for s in range(8):
        u = fourier_modes_2d(c.xyz, 100 + s)
        dt = dt_for_cfl(u, c.h, rng.uniform(2, 16))
        ud = _dev(u)
        ctx.grid_velocity(mesh, ud)
        w, t, _ = ctx.training_pairs(mesh, x, ud, dt)
        wins.append(w)
        tgts.append(t)
    W = torch.cat(wins).contiguous()
    T = torch.cat(tgts).contiguous()
    losses = ctx.train(2, W, T, batch=1024, steps=400, lr=1e-3, seed=1)
    assert losses[-20:].mean() < 0.1 * losses[:5].mean(), (losses[:5], losses[-20:])
    u = fourier_modes_2d(c.xyz, 900)
    dt = dt_for_cfl(u, c.h, 8.0)
    ud = _dev(u)
    sns = ctx.track(mesh, x, ud, dt, mode="sns")
    cnn_out = ctx.track(mesh, x, ud, dt, mode="cnn")
    torch.cuda.synchronize()
    assert torch.equal(sns["host"], cnn_out["host"])
    m_sns = sns["path_len"].double().mean().item()
    m_cnn = cnn_out["path_len"].double().mean().item()
    assert m_cnn < 0.6 * m_sns, (m_sns, m_cnn)


@pytest.mark.parametrize("n_side", [101, 301])
def test_tensor_core_grid_prediction(ctx, n_side):
    """The fused tcgen05 grid kernel against the FP64 oracle (sampled cells,
    all tile-edge and grid-edge cells included) and against the per-window
    CUDA-core engine on every cell."""
    import torch
    c = make_case("tg2d", n_side=n_side, cfl=8)
    flat = init_weights(2, 31)
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(g))
    tc = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
    win = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.predictor_engine("tc")
    ctx.predict(mesh, c.dt, out=tc)
    ctx.predictor_engine("window")
    ctx.predict(mesh, c.dt, out=win)
    ctx.predictor_engine("tc")
    ctx.device_status()
    tc, win = tc.cpu().numpy(), win.cpu().numpy()
    assert np.isfinite(tc).all()
    scale = np.abs(win).max()
    assert np.abs(tc - win).max() <= 4e-2 * scale
    # oracle on a sample: every cell of the first/last rows and columns, the
    # cells next to tile edges (multiples of 24), and random cells
    gx, gy = g
    iy, ix = np.divmod(np.arange(n_cells), gx)
    edge = (ix % 24 == 0) | (ix % 24 == 23) | (iy % 24 == 0) | (iy % 24 == 23) | \
        (ix == gx - 1) | (iy == gy - 1)
    rng = np.random.default_rng(2)
    pick = np.unique(np.concatenate([np.nonzero(edge)[0][:3000],
                                     rng.integers(0, n_cells, size=1500)]))
    U = _oracle_grid_u(om, c.u)
    s = (om.hi - om.lo) / om.grid
    w = cnn.windows(U.reshape(gy, gx, 2), pick, 2, c.dt / s)
    ref = cnn.forward(2, cnn.unpack(2, flat), w)
    # the tensor-core kernel also rounds its input window to BF16: seven
    # roundings of 2^-9 on each of two operands, 7 * 2 * 2^-9 ~ 2.7e-2 of the
    # output scale, with the worst of ~4k cells allowed 6e-2
    assert np.abs(tc[pick] - ref).max() <= 6e-2 * np.abs(ref).max()


@pytest.mark.parametrize("n_side", [101, 301])
def test_tensor_core_tile_heights_agree(ctx, n_side):
    """The tcgen05 grid kernel with tiles of 24, 13 and 8 rows and with the
    automatic choice: every cell gets the same bits whatever the height, since
    a cell's arithmetic does not depend on where the tiles cut the grid. Each
    height is also checked against the per-window engine on every cell and
    against the FP64 oracle on the cells next to its own tile edges."""
    import torch
    c = make_case("tg2d", n_side=n_side, cfl=8)
    flat = init_weights(2, 33)
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    g = mesh.info()["asg_grid"]
    om = oracle.Mesh(c.xyz, c.conn, grid=g)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(g))
    gx, gy = g
    outs = {}
    try:
        for rows in (0, 24, 13, 8):
            out = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
            ctx.predictor_tile_rows(rows)
            ctx.predict(mesh, c.dt, out=out)
            outs[rows] = out.cpu().numpy()
        win = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
        ctx.predictor_engine("window")
        ctx.predict(mesh, c.dt, out=win)
    finally:
        ctx.predictor_engine("tc")
        ctx.predictor_tile_rows(0)
    ctx.device_status()
    win = win.cpu().numpy()
    U = _oracle_grid_u(om, c.u)
    s = (om.hi - om.lo) / om.grid
    iy, ix = np.divmod(np.arange(n_cells), gx)
    for rows in (24, 13, 8):
        assert np.isfinite(outs[rows]).all(), rows
        assert np.array_equal(outs[rows].view(np.uint32), outs[24].view(np.uint32)), rows
        assert np.abs(outs[rows] - win).max() <= 4e-2 * np.abs(win).max(), rows
        edge = (ix % 24 == 0) | (ix % 24 == 23) | (iy % rows == 0) | (iy % rows == rows - 1)
        pick = np.nonzero(edge)[0][::7][:600]
        ref = cnn.forward(2, cnn.unpack(2, flat),
                          cnn.windows(U.reshape(gy, gx, 2), pick, 2, c.dt / s))
        assert np.abs(outs[rows][pick] - ref).max() <= 6e-2 * np.abs(ref).max(), rows
    assert np.array_equal(outs[0].view(np.uint32), outs[24].view(np.uint32))
    with pytest.raises(Exception):
        ctx.predictor_tile_rows(12)
    mesh.release()


# ---- the predictor grid: cells of 3^d ASG cells ----------------------------

def _oracle_pred_u(om, u_nodal):
    """FP64 P1 velocity at the predictor-cell centres, hosts by exact search."""
    cen = om.pred_centres()
    return oracle.p1_interpolate(om.conn, om.v0, om.M, u_nodal, cen, om.locate(cen))


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 101}), ("abc3d", {"n_side": 13})])
def test_predictor_grid_velocity(ctx, name, kw):
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    inf = mesh.info()
    om = oracle.Mesh(c.xyz, c.conn, grid=inf["asg_grid"], pred_stride=3)
    assert inf["pred_stride"] == 3 and inf["pred_grid"] == list(om.pgrid)
    U = torch.empty((int(np.prod(om.pgrid)), c.dim), dtype=torch.float32, device="cuda")
    ctx.grid_velocity(mesh, _dev(c.u), out=U)
    torch.cuda.synchronize()
    err = np.abs(U.cpu().numpy() - _oracle_pred_u(om, c.u)).max()
    assert err <= 5e-4 * np.abs(c.u).max(), err
    with pytest.raises(Exception):
        mesh.set_predictor_grid(2)


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 121, "cfl": 8}),
                                     ("abc3d", {"n_side": 15, "cfl": 8})])
def test_track_with_displacements_on_predictor_grid(ctx, name, kw):
    """Algorithm 2's start rule on a stride-3 predictor grid: predictor cell of
    x, x + dhat * (predictor cell size), then the ASG seed there. Bit for bit."""
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    rng = np.random.default_rng(16)
    dhat = rng.uniform(-4, 4, size=(int(np.prod(om.pgrid)), c.dim)).astype(np.float32)
    out = ctx.track_dhat(mesh, _dev(c.x), _dev(c.u), c.dt, dhat=_dev(dhat), start_out=True)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat)
    start = np.where(want["path_len"] > 0, want["start"], -1)
    for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                   ("status", want["status"]), ("start", start)):
        assert np.array_equal(got[k], ref), k


def test_training_pairs_on_predictor_grid(ctx):
    import torch
    c = make_case("tg2d", n_side=91, cfl=6)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    ctx.grid_velocity(mesh, _dev(c.u))
    win, tgt, cells = ctx.training_pairs(mesh, _dev(c.x), _dev(c.u), c.dt)
    torch.cuda.synchronize()
    assert np.array_equal(cells.cpu().numpy(), om.pred_cells(c.x))
    xp = c.x - c.u * c.dt
    assert np.array_equal(tgt.cpu().numpy(), ((xp - c.x) / om.ps).astype(np.float32))
    U = _oracle_pred_u(om, c.u)
    ref = cnn.windows(U.reshape(tuple(int(v) for v in om.pgrid[::-1]) + (2,)),
                      om.pred_cells(c.x), 2, c.dt / om.ps)
    assert np.abs(win.cpu().numpy() - ref).max() <= 5e-4 * np.abs(ref).max()


def test_tensor_core_on_predictor_grid(ctx):
    """The tcgen05 grid kernel over a stride-3 predictor grid (100 x 100 cells)
    against the per-window engine on every cell and the FP64 oracle on a sample."""
    import torch
    c = make_case("tg2d", n_side=301, cfl=8)
    flat = init_weights(2, 33)
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(om.pgrid))
    tc = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
    win = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.predictor_engine("tc")
    ctx.predict(mesh, c.dt, out=tc)
    ctx.predictor_engine("window")
    ctx.predict(mesh, c.dt, out=win)
    ctx.predictor_engine("tc")
    ctx.device_status()
    tc, win = tc.cpu().numpy(), win.cpu().numpy()
    assert np.isfinite(tc).all()
    assert np.abs(tc - win).max() <= 4e-2 * np.abs(win).max()
    rng = np.random.default_rng(3)
    pick = np.unique(np.concatenate([np.arange(0, n_cells, 97), rng.integers(0, n_cells, 800)]))
    U = _oracle_pred_u(om, c.u)
    gx, gy = (int(v) for v in om.pgrid)
    w = cnn.windows(U.reshape(gy, gx, 2), pick, 2, c.dt / om.ps)
    ref = cnn.forward(2, cnn.unpack(2, flat), w)
    assert np.abs(tc[pick] - ref).max() <= 6e-2 * np.abs(ref).max()


def test_cnn_sns_on_predictor_grid_keeps_hosts(ctx):
    """CNN-SNS with the predictor on a stride-3 grid: the same hosts as plain
    SNS (the start only changes the path), and the oracle's start rule."""
    import torch
    c = make_case("tg2d", n_side=121, cfl=8)
    flat = init_weights(2, 12)
    o = cnn.spec(2)
    fc2 = sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in o[:-1])
    flat[fc2:] *= 0.25
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    out = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode="cnn", start_out=True)
    dhat = torch.empty((int(np.prod(mesh.info()["pred_grid"])), 2), dtype=torch.float32,
                       device="cuda")
    ctx.predict(mesh, c.dt, out=dhat)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat.cpu().numpy())
    plain = om.track(c.x, c.u, c.dt, mode="sns")
    assert np.array_equal(got["host"], plain["host"])
    for k in ("host", "path_len", "status"):
        assert np.array_equal(got[k], want[k]), k


@pytest.mark.parametrize("n_side,stride", [(13, 1), (31, 3), (53, 1)])
def test_tile_engine_3d_matches_windows(ctx, n_side, stride):
    """The 3-D fully convolutional tile engine against the per-window engine on
    every predictor cell (one tile, and several tiles with a ragged last one),
    and the per-window engine against the FP64 oracle on a sample."""
    import torch
    c = make_case("abc3d", n_side=n_side, cfl=6)
    flat = init_weights(3, 41)
    ctx.load_predictor(3, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=stride)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(om.pgrid))
    tile = torch.full((n_cells, 3), float("nan"), dtype=torch.float32, device="cuda")
    win = torch.full((n_cells, 3), float("nan"), dtype=torch.float32, device="cuda")
    try:
        ctx.predictor_engine("tiles")
        ctx.predict(mesh, c.dt, out=tile)
        ctx.predictor_engine("window")
        ctx.predict(mesh, c.dt, out=win)
    finally:
        ctx.predictor_engine("tc")
    torch.cuda.synchronize()
    tile, win = tile.cpu().numpy(), win.cpu().numpy()
    assert np.isfinite(tile).all()
    # the same layers on the same BF16 operands, but the tile engine's
    # convolutions add their K range as four partial sums: the FP32
    # reassociation can move an activation across a BF16 rounding boundary
    # before the next layer, a 2^-8 relative change of that input (1.2e-3 of
    # the output scale measured); the bound leaves room for a few such flips
    assert np.abs(tile - win).max() <= 1e-2 * np.abs(win).max()
    rng = np.random.default_rng(7)
    pick = np.unique(np.concatenate([[0, n_cells - 1], rng.integers(0, n_cells, 200)]))
    U = _oracle_pred_u(om, c.u)
    w = cnn.windows(U.reshape(tuple(int(v) for v in om.pgrid[::-1]) + (3,)), pick, 3,
                    c.dt / om.ps)
    ref = cnn.forward(3, cnn.unpack(3, flat), w)
    assert np.abs(win[pick] - ref).max() <= 5e-2 * np.abs(ref).max()


def test_cnn_sns_3d_on_tiles_keeps_hosts(ctx):
    """3-D CNN-SNS through the tile engine: hosts equal plain SNS and the
    oracle's start rule, bit for bit, on the engine's own predictions."""
    import torch
    c = make_case("abc3d", n_side=21, cfl=8)
    flat = init_weights(3, 12)
    o = cnn.spec(3)
    fc2 = sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in o[:-1])
    flat[fc2:] *= 0.25
    ctx.load_predictor(3, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(3)
    out = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode="cnn")
    dhat = torch.empty((int(np.prod(mesh.info()["pred_grid"])), 3), dtype=torch.float32,
                       device="cuda")
    ctx.predict(mesh, c.dt, out=dhat)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=3)
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat.cpu().numpy())
    plain = om.track(c.x, c.u, c.dt, mode="sns")
    assert np.array_equal(got["host"], plain["host"])
    for k in ("host", "path_len", "status"):
        assert np.array_equal(got[k], want[k]), k


def test_full_size_cnn_sns_parity(ctx):
    """The 1001 x 1001 Taylor-Green workload at CFL 8 with the predictor on
    the stride-5 grid (the benchmark's configuration): the oracle, given the
    device's predicted displacements, takes the same starts, paths, statuses
    and hosts on every particle, and the hosts are plain SNS's."""
    import torch
    c = make_case("tg2d", cfl=8)
    flat = init_weights(2, 12)
    o = cnn.spec(2)
    fc2 = sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in o[:-1])
    flat[fc2:] *= 0.25
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(5)
    out = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode="cnn", start_out=True)
    dhat = torch.empty((int(np.prod(mesh.info()["pred_grid"])), 2), dtype=torch.float32,
                       device="cuda")
    ctx.predict(mesh, c.dt, out=dhat)
    torch.cuda.synchronize()
    got = {k: v.cpu().numpy() for k, v in out.items()}
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=5)
    want = om.track(c.x, c.u, c.dt, mode="cnn", dhat=dhat.cpu().numpy())
    start = np.where(want["path_len"] > 0, want["start"], -1)
    for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                   ("status", want["status"]), ("start", start)):
        bad = np.nonzero(got[k] != ref)[0]
        assert bad.size == 0, (k, bad.size, bad[:5])
    plain = om.track(c.x, c.u, c.dt, mode="sns")
    assert np.array_equal(got["host"], plain["host"])
    mesh.release()


# ---- direct oracle parity of every grid engine ------------------------------

@pytest.mark.parametrize("engine", ["tc", "tiles"])
@pytest.mark.parametrize("n_side,stride", [(13, 1), (31, 3)])
def test_tile_engine_3d_matches_oracle_on_every_cell(ctx, n_side, stride, engine):
    """The 3-D fully convolutional engines (the tcgen05 kernel, and the tile
    engine on CUDA cores) against the FP64 forward pass (oracle.cnn.forward on
    oracle windows of the oracle's grid velocity) on every predictor cell.
    Tolerance: both round the input window and every layer's operands to BF16
    (relative 2^-9 each): five layers x two operands plus the input,
    11 x 2^-9 ~ 2.1e-2 of the output scale; the bound allows the worst cell
    5e-2, the 2-D bound's margin (4e-2 for 7 roundings there) scaled alike."""
    import torch
    c = make_case("abc3d", n_side=n_side, cfl=6)
    flat = init_weights(3, 41)
    ctx.load_predictor(3, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=stride)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(om.pgrid))
    tile = torch.full((n_cells, 3), float("nan"), dtype=torch.float32, device="cuda")
    try:
        ctx.predictor_engine(engine)
        ctx.predict(mesh, c.dt, out=tile)
        ctx.device_status()
    finally:
        ctx.predictor_engine("tc")
    torch.cuda.synchronize()
    tile = tile.cpu().numpy()
    U = _oracle_pred_u(om, c.u)
    cells = np.arange(n_cells)
    w = cnn.windows(U.reshape(tuple(int(v) for v in om.pgrid[::-1]) + (3,)), cells, 3,
                    c.dt / om.ps)
    ref = cnn.forward(3, cnn.unpack(3, flat), w)
    assert np.isfinite(tile).all()
    err = np.abs(tile - ref).max()
    assert err <= 5e-2 * np.abs(ref).max(), (err, np.abs(ref).max())
    mesh.release()


def test_tensor_core_at_the_benchmark_configuration(ctx):
    """The tcgen05 grid kernel exactly as the benchmark runs it: the 1001^2
    Taylor-Green mesh, predictor grid stride 5 (200 x 200 cells), automatic
    tile height (13 rows: 144 tiles), against the FP64 forward pass on every
    cell next to a tile edge or the grid edge and on 3000 random cells. The
    bound is the 2-D one (6e-2 of the output scale: the BF16 input window and
    six layers' BF16 operands)."""
    import torch
    c = make_case("tg2d", cfl=8)
    flat = init_weights(2, 31)
    ctx.load_predictor(2, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(5)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"], pred_stride=5)
    gx, gy = (int(v) for v in om.pgrid)
    assert (gx, gy) == (200, 200)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = gx * gy
    tc = torch.full((n_cells, 2), float("nan"), dtype=torch.float32, device="cuda")
    ctx.predictor_engine("tc")
    ctx.predictor_tile_rows(0)
    ctx.predict(mesh, c.dt, out=tc)
    ctx.device_status()
    tc = tc.cpu().numpy()
    assert np.isfinite(tc).all()
    th = 13
    iy, ix = np.divmod(np.arange(n_cells), gx)
    edge = ((ix % 24 == 0) | (ix % 24 == 23) | (iy % th == 0) | (iy % th == th - 1) |
            (ix == gx - 1) | (iy == gy - 1))
    rng = np.random.default_rng(8)
    pick = np.unique(np.concatenate([np.nonzero(edge)[0], rng.integers(0, n_cells, 3000)]))
    U = _oracle_pred_u(om, c.u)
    w = cnn.windows(U.reshape(gy, gx, 2), pick, 2, c.dt / om.ps)
    ref = cnn.forward(2, cnn.unpack(2, flat), w)
    err = np.abs(tc[pick] - ref).max()
    assert err <= 6e-2 * np.abs(ref).max(), (err, np.abs(ref).max())
    mesh.release()


@pytest.mark.parametrize("dim", [2, 3])
def test_adam_steps_against_the_oracle(ctx, dim):
    """Five training steps on the device against oracle.cnn.Adam. With a
    batch of one pair the step's gradient is, bit for bit, the one
    cs_predictor_grad returns at the step's weights (no shuffle, no
    reordered sums); the oracle's Adam takes those gradients from the same
    start and keeps its own FP64 moments and bias corrections. The device
    updates its FP32 master weights with FP32 arithmetic: each step is off by
    a few units in the last place of a 1e-3 update and of weights of order
    0.1, so the weights agree to 1e-7 after every step, with the moments of
    all five steps carried on both sides."""
    rng = np.random.default_rng(60 + dim)
    flat = init_weights(dim, 9)
    ctx.load_predictor(dim, flat)
    S = cnn.patch_size(dim)
    win = _dev(rng.standard_normal((1, dim) + (S,) * dim).astype(np.float32))
    tgt = _dev(rng.standard_normal((1, dim)).astype(np.float32))
    opt = cnn.Adam(flat.size, lr=1e-3)
    w_ref = flat.astype(np.float32).astype(np.float64)
    moved = np.zeros(flat.size, dtype=bool)
    for step in range(5):
        g, _ = ctx.predictor_grad(dim, win, tgt)
        g = g.cpu().numpy().astype(np.float64)
        w_ref = opt.step(w_ref, g)
        ctx.train(dim, win, tgt, batch=1, steps=1, lr=1e-3, seed=step)
        w_dev = ctx.save_predictor(dim).astype(np.float64)
        assert np.allclose(w_dev, w_ref, rtol=0, atol=1e-7), (step, np.abs(w_dev - w_ref).max())
        moved |= w_dev != flat
        # the device follows the oracle's moments: continue from its own weights
        w_ref = w_dev.copy()
    assert opt.t == 5 and moved.mean() > 0.5


@pytest.mark.parametrize("dim", [2, 3])
def test_training_is_bit_reproducible(ctx, dim):
    """The K splits of the training GEMMs are summed in a fixed order, so a
    gradient, and a whole training run from the same weights and seed, give
    the same bits every time."""
    rng = np.random.default_rng(80 + dim)
    S = cnn.patch_size(dim)
    B = 1024 if dim == 2 else 256
    win = _dev(rng.standard_normal((4 * B, dim) + (S,) * dim).astype(np.float32))
    tgt = _dev(rng.standard_normal((4 * B, dim)).astype(np.float32))
    flat = init_weights(dim, 19)
    runs = []
    for _ in range(2):
        ctx.load_predictor(dim, flat)
        g, loss = ctx.predictor_grad(dim, win[:B].contiguous(), tgt[:B].contiguous())
        losses = ctx.train(dim, win, tgt, batch=B, steps=6, lr=1e-3, seed=5)
        runs.append((g.cpu().numpy(), loss, losses, ctx.save_predictor(dim)))
    (g0, l0, ls0, w0), (g1, l1, ls1, w1) = runs
    assert np.array_equal(g0.view(np.uint32), g1.view(np.uint32)) and l0 == l1
    assert np.array_equal(ls0.view(np.uint32), ls1.view(np.uint32))
    assert np.array_equal(w0.view(np.uint32), w1.view(np.uint32))


@pytest.mark.parametrize("n_side,stride", [(29, 1), (61, 3)])
def test_tensor_core_3d_tile_sides_agree(ctx, n_side, stride):
    """The 3-D tcgen05 grid kernel with output tiles of side 4, 3 and 2 and
    the automatic choice: every cell gets the same bits (a cell's MMAs and
    their order do not depend on where the tiles cut the grid), all finite,
    and against the CUDA-core tile engine within the BF16 bound (1e-2 of the
    output scale: the same roundings, FP32 sums in another order)."""
    import torch
    c = make_case("abc3d", n_side=n_side, cfl=8)
    flat = init_weights(3, 43)
    ctx.load_predictor(3, flat)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    ctx.grid_velocity(mesh, _dev(c.u))
    n_cells = int(np.prod(mesh.info()["pred_grid"]))
    outs = {}
    try:
        for side in (0, 4, 3, 2):
            o = torch.full((n_cells, 3), float("nan"), dtype=torch.float32, device="cuda")
            ctx.predictor_tile3(side)
            ctx.predict(mesh, c.dt, out=o)
            outs[side] = o.cpu().numpy()
        tiles = torch.full((n_cells, 3), float("nan"), dtype=torch.float32, device="cuda")
        ctx.predictor_engine("tiles")
        ctx.predict(mesh, c.dt, out=tiles)
    finally:
        ctx.predictor_engine("tc")
        ctx.predictor_tile3(0)
    ctx.device_status()
    tiles = tiles.cpu().numpy()
    for side in (0, 3, 2):
        assert np.isfinite(outs[side]).all(), side
        assert np.array_equal(outs[side].view(np.uint32), outs[4].view(np.uint32)), side
    assert np.abs(outs[4] - tiles).max() <= 1e-2 * np.abs(tiles).max()
    with pytest.raises(Exception):
        ctx.predictor_tile3(5)
    mesh.release()


@pytest.mark.parametrize("dim", [2, 3])
def test_tensor_core_gradients_at_training_batch(ctx, dim):
    """The training GEMMs on the tensor cores at a batch that splits the weight
    gradients' long K (the batch positions) over CTAs: every layer's gradient
    against the FP64 backward within the BF16 bound of the per-layer test
    (1.5e-1 relative for the deepest layer, 5e-2 for the others), and the loss
    within 4e-2."""
    rng = np.random.default_rng(70 + dim)
    flat = init_weights(dim, 17).astype(np.float64)
    flat += 0.02 * rng.standard_normal(flat.size)
    flat = flat.astype(np.float32)
    ctx.load_predictor(dim, flat)
    S = cnn.patch_size(dim)
    B = 2048 if dim == 2 else 512
    win = rng.standard_normal((B, dim) + (S,) * dim).astype(np.float32)
    tgt = rng.standard_normal((B, dim)).astype(np.float32)
    params = cnn.unpack(dim, flat)
    ref, acts = cnn.forward(dim, params, win.astype(np.float64), keep=True)
    gref = cnn.pack(cnn.backward(dim, params, acts, ref, tgt.astype(np.float64)))
    g, loss = ctx.predictor_grad(dim, _dev(win), _dev(tgt))
    ctx.device_status()
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss - cnn.mse(ref, tgt)) <= 4e-2 * cnn.mse(ref, tgt)
    o = 0
    for li, (_, ws, bs) in enumerate(cnn.spec(dim)):
        n = int(np.prod(ws)) + int(np.prod(bs))
        a, b = g[o:o + n], gref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel <= (1.5e-1 if li == 0 else 5e-2), (li, rel)
        o += n


@pytest.mark.parametrize("name,kw,stride", [("tg2d", {"n_side": 201}, 1), ("abc3d", {"n_side": 25}, 1)])
def test_a_wait_that_runs_out_ends_the_kernel_with_cs_edevice(ctx, name, kw, stride):
    """The bounded waits of the tensor-core predictor kernels: with the test
    hook on, each kernel first waits (about 17 ms) for a device flag that
    nothing sets; the wait runs out, the kernel ends through its abort path
    (no MMA issued, TMEM freed) and cs_device_status reports CS_EDEVICE. The
    context stays usable: with the hook off the same prediction gives the bits
    it gave before, and the device status is clean again."""
    import time
    import torch
    import paper_2412_18379_gb300 as cs
    c = make_case(name, **kw)
    ctx.load_predictor(c.dim, init_weights(c.dim, 3))
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    mesh.set_predictor_grid(stride)
    ctx.grid_velocity(mesh, _dev(c.u))
    cells = int(np.prod(mesh.info()["pred_grid"]))
    before = torch.empty((cells, c.dim), dtype=torch.float32, device="cuda")
    ctx.predict(mesh, c.dt, out=before)
    ctx.device_status()
    held = torch.full((cells, c.dim), float("nan"), dtype=torch.float32, device="cuda")
    ctx.debug_hold_predictor(True)
    try:
        t0 = time.perf_counter()
        ctx.predict(mesh, c.dt, out=held)
        with pytest.raises(cs.CsError) as e:
            ctx.device_status()
        assert e.value.code == -8 and "gave up" in str(e.value)
        assert time.perf_counter() - t0 < 30.0
    finally:
        ctx.debug_hold_predictor(False)
    ctx.device_status()                      # the flag was read and cleared
    after = torch.full((cells, c.dim), float("nan"), dtype=torch.float32, device="cuda")
    ctx.predict(mesh, c.dt, out=after)
    ctx.device_status()
    assert np.array_equal(before.cpu().numpy().view(np.uint32), after.cpu().numpy().view(np.uint32))
    mesh.release()


@pytest.mark.parametrize("rows", [24, 13, 8])
def test_fused_resample_gives_the_resample_kernels_bits(ctx, rows):
    """CNN-SNS on the mesh nodes in 2-D resamples the nodal velocity inside
    the tensor-core predictor as it loads its tiles. On a 400^2 predictor
    grid (289 to 850 tiles: CTAs take several, so both the first-tile and the
    loader warp's path run), the grid velocity it stores and the predictions
    it starts the walks from must equal, bit for bit, those of the separate
    resample kernel followed by the prediction."""
    import torch
    c = make_case("tg2d", n_side=401, cfl=8)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    ctx.load_predictor(2, init_weights(2, 41))
    ctx.predictor_tile_rows(rows)
    try:
        cells = int(np.prod(mesh.info()["pred_grid"]))
        fused = ctx.track(mesh, _dev(c.x), _dev(c.u), c.dt, mode="cnn", start_out=True)
        a = torch.empty((cells, 2), dtype=torch.float32, device="cuda")
        ctx.predict(mesh, c.dt, out=a)            # from the grid velocity the track stored
        ctx.grid_velocity(mesh, _dev(c.u))         # the resample kernel
        b = torch.empty((cells, 2), dtype=torch.float32, device="cuda")
        ctx.predict(mesh, c.dt, out=b)
        ref = ctx.track_dhat(mesh, _dev(c.x), _dev(c.u), c.dt, dhat=b, start_out=True)
        torch.cuda.synchronize()
        ctx.device_status()
        assert torch.equal(a, b)
        for k in ("start", "host", "path_len", "status"):
            assert torch.equal(fused[k], ref[k]), k
    finally:
        ctx.predictor_tile_rows(0)
