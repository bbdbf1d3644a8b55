"""The paper's classifier predictor (Sec. 2.3, Eq. 7-8) on the GPU against
the FP64 oracle (oracle/classifier.py), through the C ABI.

Integer and FP64 work is compared bit for bit: the pooled-centroid windows
and offsets (FP64 formulas rounded once to float32), the labels from plain
SNS hosts, the start element of a given class, and the hosts, paths and
status of the walk from the classifier's starts.

Tolerances of the network. With FP32 operands (cs_predictor_precision 0)
the logits agree with the FP64 forward to 1e-4 of their scale (FP32
accumulation over at most 864 * 27 terms per layer), and every layer's
gradient to 1e-3 relative in norm (weight gradients sum over the batch's
B * W^dim positions). With BF16 operands (the default arithmetic) each of
the four layers on the convolution path rounds its inputs and weights once:
about 4 * 2 * 2^-9 ~ 1.6e-2 of the scale, allowed 4e-2; gradients pass
through up to 2 * 4 rounded operands and the ReLU gates of a forward pass
off by ~1e-2: 1.5e-1 relative for the first convolution, 8e-2 for the
others. The class is an argmax over logits computed in different
precisions: the device's class must be one whose FP64 logit lies within
that tolerance of the FP64 maximum, and the start is then checked bit for
bit as the oracle's start of the device's class.
"""

import numpy as np
import pytest

import oracle
from oracle import classifier as ocls
from workloads import make_case
from workloads.fields import fourier_modes_2d, fourier_modes_3d, dt_for_cfl
from workloads.weights import init_classifier, classifier_layer_shapes

pytestmark = pytest.mark.gpu

CASES = [("tg2d", {"n_side": 41}), ("abc3d", {"n_side": 9})]


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
    return torch.from_numpy(np.array(a, copy=True, order="C")).cuda()


def _unflatten(dim, flat):
    out, o = [], 0
    for ws, bs in classifier_layer_shapes(dim):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((flat[o:o + nw].astype(np.float64).reshape(ws),
                    flat[o + nw:o + nw + nb].astype(np.float64)))
        o += nw + nb
    assert o == flat.size
    return out


def _flatten(params):
    return np.concatenate([np.concatenate([w.ravel(), b.ravel()]) for w, b in params])


def _setup(ctx, name, kw):
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    return c, mesh, om


def _points(om, n, seed, outside=0.0):
    """Departure points spread over the box (a share `outside` beyond it)."""
    rng = np.random.default_rng(seed)
    ext = om.hi - om.lo
    p = om.lo + rng.random((n, om.dim)) * ext
    k = int(outside * n)
    if k:
        p[:k] = om.lo + (rng.random((k, om.dim)) * 1.4 - 0.2) * ext
    if n - k >= 6:
        # cell faces and the box corners
        s = ext / om.grid
        p[k:k + 4] = om.lo + np.floor((p[k:k + 4] - om.lo) / s) * s
        p[k + 4] = om.lo
        p[k + 5] = om.hi
    return p


def test_classifier_sizes(ctx):
    for dim in (2, 3):
        assert ctx.classifier_size(dim) == init_classifier(dim, 0).size
        assert ctx.classifier_window(dim) == ocls.window_size(dim)
    assert ctx.classifier_size(4) == 0


@pytest.mark.parametrize("name,kw", CASES)
def test_features_match_oracle_bit_for_bit(ctx, name, kw):
    """The pooled-centroid windows and offsets are the oracle's FP64 values
    rounded once to float32, for points inside, on cell faces and outside
    the mesh box (windows reaching past the grid take the padding centres)."""
    import torch
    c, mesh, om = _setup(ctx, name, kw)
    xp = _points(om, 700, 3, outside=0.2)
    win, off = ctx.classifier_features(mesh, _dev(xp))
    torch.cuda.synchronize()
    rwin, roff, _ = ocls.features(om, xp)
    assert np.array_equal(win.cpu().numpy(), rwin.astype(np.float32))
    assert np.array_equal(off.cpu().numpy(), roff.astype(np.float32))


@pytest.mark.parametrize("name,kw", CASES)
def test_labels_and_pairs_match_oracle(ctx, name, kw):
    """Labels from plain SNS hosts, bit for bit, through cs_classifier_labels
    and through cs_classifier_pairs (departure points, walk and labels on the
    device); -1 where the host is -1."""
    import torch
    c, mesh, om = _setup(ctx, name, kw)
    ref = om.track(c.x, c.u, c.dt)
    xp_ref = ref["xp"]
    host = ref["host"].astype(np.int32)
    want = ocls.labels(om, xp_ref, host)
    lab = ctx.classifier_labels(mesh, _dev(xp_ref), _dev(host))
    xp, lab2 = ctx.classifier_pairs(mesh, _dev(c.x), _dev(c.u), c.dt)
    torch.cuda.synchronize()
    assert np.array_equal(xp.cpu().numpy(), xp_ref)
    assert np.array_equal(lab.cpu().numpy(), want)
    assert np.array_equal(lab2.cpu().numpy(), want)
    xpd = ctx.departure(mesh, _dev(c.x), _dev(c.u), c.dt)
    torch.cuda.synchronize()
    assert np.array_equal(xpd.cpu().numpy(), oracle.departure(c.x, c.u, c.dt))


def _grad_check(ctx, mesh, om, flat, xp, labels, bf16):
    params = _unflatten(om.dim, flat)
    win, off, _ = ocls.features(om, xp)
    ctx.predictor_precision(bf16)
    try:
        ctx.load_classifier(om.dim, flat)
        H = ctx.classifier_forward(mesh, _dev(xp)).cpu().numpy()
        g, loss = ctx.classifier_grad(mesh, _dev(xp), _dev(labels.astype(np.int32)))
        g = g.cpu().numpy().astype(np.float64)
    finally:
        ctx.predictor_precision(True)
    Href, P, keep = ocls.forward(params, win, off, keep=True)
    scale = np.abs(Href).max()
    ftol = 4e-2 if bf16 else 1e-4
    assert np.abs(H - Href).max() <= ftol * scale, np.abs(H - Href).max() / scale
    ce = ocls.cross_entropy(P, labels)
    assert abs(loss - ce) <= (4e-2 if bf16 else 1e-4) * max(ce, 1.0), (loss, ce)
    gref = _flatten(ocls.backward(params, P, labels, keep))
    o = 0
    for li, (ws, bs) in enumerate(classifier_layer_shapes(om.dim)):
        n = int(np.prod(ws)) + int(np.prod(bs))
        a, b = g[o:o + n], gref[o:o + n]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        tol = (1.5e-1 if li == 0 else 8e-2) if bf16 else 1e-3
        assert rel <= tol, (li, ws, rel)
        o += n
    return H, Href


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("name,kw", CASES)
def test_forward_and_gradient_match_oracle(ctx, name, kw, bf16):
    """Logits, cross-entropy and every layer's gradient against the FP64
    forward and backward, with FP32 and with BF16 operands."""
    c, mesh, om = _setup(ctx, name, kw)
    dim = om.dim
    B = 200 if dim == 2 else 48
    xp = _points(om, B, 5, outside=0.1)
    rng = np.random.default_rng(6)
    flat = init_classifier(dim, 3).astype(np.float64)
    flat += 0.02 * rng.standard_normal(flat.size)      # non-zero biases
    flat = flat.astype(np.float32)
    labels = rng.integers(0, ocls.window_size(dim) ** dim, size=B)
    _grad_check(ctx, mesh, om, flat, xp, labels, bf16)


@pytest.mark.parametrize("name,kw,n", [("tg2d", {"n_side": 41}, 70000),
                                        ("abc3d", {"n_side": 9}, 36000)])
def test_inference_over_several_chunks(ctx, name, kw, n):
    """Inference runs module 1 fused on the tensor cores, in chunks of 32768
    (2-D) or 16384 (3-D) particles: logits of a batch spanning three chunks,
    with a ragged last one, against the FP64 forward on a sample of rows
    (every chunk's first and last row included), within the BF16 bound."""
    c, mesh, om = _setup(ctx, name, kw)
    dim = om.dim
    xp = _points(om, n, 21, outside=0.05)
    flat = init_classifier(dim, 11)
    ctx.load_classifier(dim, flat)
    H = ctx.classifier_forward(mesh, _dev(xp)).cpu().numpy()
    chunk = 32768 if dim == 2 else 16384
    rng = np.random.default_rng(22)
    rows = np.unique(np.concatenate([rng.choice(n, 150 if dim == 2 else 40, replace=False),
                                     np.arange(0, n, chunk), np.arange(chunk - 1, n, chunk),
                                     [n - 1]]))
    win, off, _ = ocls.features(om, xp[rows])
    Href, _ = ocls.forward(_unflatten(dim, flat), win, off)
    assert np.abs(H[rows] - Href).max() <= 4e-2 * np.abs(Href).max()
    assert np.isfinite(H).all()


@pytest.mark.parametrize("name,kw", CASES)
def test_rows_without_label_count_for_nothing(ctx, name, kw):
    """Rows with a label outside [0, W^dim) add nothing to the loss or the
    gradient: the result is that of the labelled rows alone."""
    c, mesh, om = _setup(ctx, name, kw)
    dim = om.dim
    B = 64 if dim == 2 else 16
    xp = _points(om, B, 8)
    rng = np.random.default_rng(9)
    labels = rng.integers(0, ocls.window_size(dim) ** dim, size=B).astype(np.int32)
    ctx.load_classifier(dim, init_classifier(dim, 4))
    g_all, l_all = ctx.classifier_grad(mesh, _dev(xp[: B // 2]), _dev(labels[: B // 2]))
    lab = labels.copy()
    lab[B // 2:] = -1
    lab[-1] = ocls.window_size(dim) ** dim       # one past the last class
    g_mix, l_mix = ctx.classifier_grad(mesh, _dev(xp), _dev(lab))
    assert np.allclose(g_mix.cpu().numpy(), g_all.cpu().numpy(), rtol=1e-5, atol=1e-7)
    assert abs(l_mix - l_all) <= 1e-5 * l_all


@pytest.mark.parametrize("name,kw", CASES)
def test_start_matches_oracle(ctx, name, kw):
    """K_p (Eq. 8): the device's class is an FP64 argmax within the BF16
    tolerance, and the start of that class is the oracle's, bit for bit,
    including the fallback to the given plain start where the predicted cell
    lies outside the grid or its centre outside the mesh."""
    import torch
    c, mesh, om = _setup(ctx, name, kw)
    dim = om.dim
    n = 400 if dim == 2 else 120
    xp = _points(om, n, 11, outside=0.15)
    flat = init_classifier(dim, 5)
    ctx.load_classifier(dim, flat)
    H = ctx.classifier_forward(mesh, _dev(xp))
    fallback = np.arange(n, dtype=np.int32) % om.n_e
    start, cls = ctx.classifier_start(mesh, _dev(xp), H, fallback=_dev(fallback))
    torch.cuda.synchronize()
    start, cls = start.cpu().numpy(), cls.cpu().numpy()
    win, off, _ = ocls.features(om, xp)
    Href, _ = ocls.forward(_unflatten(dim, flat), win, off)
    assert (cls >= 0).all()
    top = Href.max(axis=1)
    picked = Href[np.arange(n), cls]
    assert (top - picked <= 4e-2 * np.abs(Href).max()).all()
    assert (cls == Href.argmax(axis=1)).mean() > 0.9
    want = ocls.start_elements(om, xp, cls)
    want = np.where(want >= 0, want, fallback)
    assert np.array_equal(start, want)
    assert (want == fallback).any() and (want != fallback).any()


def test_start_ties_rows_without_class_and_node_fallback(ctx):
    """Hand-set logits: equal maxima give the lowest class; a row of NaN or
    -inf has no class (class -1, the fallback start); without a fallback
    array the mesh nodes' plain starts are used."""
    import torch
    c, mesh, om = _setup(ctx, "tg2d", {"n_side": 41})
    n = om.n_v
    ncls = 81
    H = np.zeros((n, ncls), dtype=np.float32)
    H[:, 7] = 1.0
    H[:, 30] = 1.0            # tie with class 7
    H[0, :] = np.nan
    H[1, :] = -np.inf
    H[2, 40] = 2.0
    xp = c.xyz.astype(np.float64)
    start, cls = ctx.classifier_start(mesh, _dev(xp), _dev(H))
    torch.cuda.synchronize()
    start, cls = start.cpu().numpy(), cls.cpu().numpy()
    assert cls[0] == -1 and cls[1] == -1 and cls[2] == 40
    assert (cls[3:] == 7).all()
    want = ocls.start_elements(om, xp, np.maximum(cls, 0))
    want[:2] = -1
    plain = mesh.node_start_elements()
    want = np.where(want >= 0, want, plain)
    assert np.array_equal(start, want)


@pytest.mark.parametrize("name,kw", CASES)
def test_track_with_classifier_keeps_hosts(ctx, name, kw):
    """CNN-SNS through the classifier: the starts are cs_classifier_start's
    (plain start as fallback), and the walk from them gives the oracle's
    hosts, paths and status bit for bit; hosts equal plain SNS's."""
    import torch
    c, mesh, om = _setup(ctx, name, kw)
    ctx.load_classifier(om.dim, init_classifier(om.dim, 6))
    out = ctx.track_classifier(mesh, _dev(c.x), _dev(c.u), c.dt, start_out=True)
    torch.cuda.synchronize()
    xp = oracle.departure(c.x, c.u, c.dt)
    H = ctx.classifier_forward(mesh, _dev(xp))
    st, _ = ctx.classifier_start(mesh, _dev(xp), H)
    torch.cuda.synchronize()
    starts = out["start"].cpu().numpy()
    assert np.array_equal(starts, st.cpu().numpy())
    ref = om.track(c.x, c.u, c.dt, start=starts)
    sns = om.track(c.x, c.u, c.dt)
    for k in ("host", "path_len", "status"):
        assert np.array_equal(out[k].cpu().numpy(), ref[k]), k
    assert np.array_equal(ref["host"], sns["host"])


@pytest.mark.parametrize("dim", [2, 3])
def test_adam_steps_against_the_oracle(ctx, dim):
    """Four training steps on a batch of one pair against oracle.cnn.Adam fed
    with the device's own gradients at each step's parameters (FP32 device
    arithmetic against FP64 moments). Each step's 1e-3 update agrees to a few
    units in its last place, and the FP32 master weight is rounded once more:
    the offset branch's first layer (fan-in dim, He-normal weights up to ~4)
    holds weights whose float32 spacing is 4.8e-7, so the bound is 1e-7 plus
    one float32 unit in the last place of the weight (2^-23 relative)."""
    from oracle import cnn
    name, kw = CASES[dim - 2]
    c, mesh, om = _setup(ctx, name, kw)
    xp = _dev(_points(om, 1, 12))
    lab = _dev(np.array([17], dtype=np.int32))
    flat = init_classifier(dim, 7)
    ctx.load_classifier(dim, flat)
    opt = cnn.Adam(flat.size, lr=1e-3)
    w_ref = flat.astype(np.float64)
    moved = np.zeros(flat.size, dtype=bool)
    for step in range(4):
        g, _ = ctx.classifier_grad(mesh, xp, lab)
        w_ref = opt.step(w_ref, g.cpu().numpy().astype(np.float64))
        ctx.train_classifier(mesh, xp, lab, batch=1, steps=1, lr=1e-3, seed=step)
        w_dev = ctx.save_classifier(dim).astype(np.float64)
        bound = 1e-7 + 2.0 ** -23 * np.abs(w_ref)
        assert (np.abs(w_dev - w_ref) <= bound).all(), (step, np.abs(w_dev - w_ref).max())
        moved |= w_dev != flat
        w_ref = w_dev.copy()
    assert moved.mean() > 0.3


@pytest.mark.parametrize("dim", [2, 3])
def test_training_is_bit_reproducible(ctx, dim):
    """Fixed-order reductions everywhere (GEMM K splits, column sums, the
    softmax block): two training runs from the same parameters and seed give
    the same losses and parameters bit for bit."""
    name, kw = CASES[dim - 2]
    c, mesh, om = _setup(ctx, name, kw)
    n = 600 if dim == 2 else 160
    xp = _dev(_points(om, n, 13))
    rng = np.random.default_rng(14)
    lab = _dev(rng.integers(0, ocls.window_size(dim) ** dim, size=n).astype(np.int32))
    flat = init_classifier(dim, 8)
    runs = []
    for _ in range(2):
        ctx.load_classifier(dim, flat)
        losses = ctx.train_classifier(mesh, xp, lab, batch=n // 3, steps=5, lr=1e-3, seed=2)
        runs.append((losses, ctx.save_classifier(dim)))
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_training_lowers_the_loss_and_shortens_walks(ctx):
    """Trained on pairs from random 8-mode fields (Sec. 2.3: the tracking
    produces its own training data), the classifier's loss falls and, on a
    held-out field, its starts shorten the walk against plain SNS while the
    hosts stay those of plain SNS."""
    import torch
    c = make_case("tg2d", n_side=121)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    h = 1.0 / 120
    xs, labs = [], []
    for seed in range(4):
        u = fourier_modes_2d(c.xyz, seed=200 + seed)
        dt = dt_for_cfl(u, h, 3.0)
        xp, lab = ctx.classifier_pairs(mesh, _dev(c.xyz), _dev(u), dt)
        xs.append(xp)
        labs.append(lab)
    xp = torch.cat(xs)
    lab = torch.cat(labs)
    ctx.load_classifier(2, init_classifier(2, 9))
    losses = ctx.train_classifier(mesh, xp, lab, batch=1024, steps=400, lr=1e-3, seed=1)
    assert losses[-20:].mean() < 0.5 * losses[:5].mean(), (losses[:5], losses[-20:])
    u = fourier_modes_2d(c.xyz, seed=999)
    dt = dt_for_cfl(u, h, 3.0)
    out = ctx.track_classifier(mesh, _dev(c.xyz), _dev(u), dt)
    sns = ctx.track(mesh, _dev(c.xyz), _dev(u), dt)
    torch.cuda.synchronize()
    assert np.array_equal(out["host"].cpu().numpy(), sns["host"].cpu().numpy())
    p_cls = out["path_len"].double().mean().item()
    p_sns = sns["path_len"].double().mean().item()
    assert p_cls < 0.7 * p_sns, (p_cls, p_sns)


def test_empty_and_refused_calls(ctx):
    """n = 0 is a no-op; without a classifier of the mesh's dimension the
    network calls are refused with CS_ENOPRED; bad sizes with CS_EINVAL."""
    import paper_2412_18379_gb300 as cs
    import torch
    c = make_case("tg2d", n_side=21)
    fresh = cs.Context(0)
    try:
        mesh = fresh.upload_mesh(c.xyz, c.conn)
        empty = torch.empty((0, 2), dtype=torch.float64, device="cuda")
        xp = _dev(c.xyz.astype(np.float64))
        with pytest.raises(cs.CsError) as e:
            fresh.classifier_forward(mesh, xp)
        assert e.value.code == -7
        with pytest.raises(cs.CsError) as e:
            fresh.track_classifier(mesh, _dev(c.x), _dev(c.u), c.dt)
        assert e.value.code == -7
        with pytest.raises(ValueError):
            fresh.load_classifier(2, np.zeros(10, dtype=np.float32))
        win, off = fresh.classifier_features(mesh, empty)
        assert win.shape == (0, 2, 9, 9) and off.shape == (0, 2)
        fresh.load_classifier(2, init_classifier(2, 0))
        assert fresh.classifier_forward(mesh, empty).shape == (0, 81)
        with pytest.raises(cs.CsError) as e:
            fresh.train_classifier(mesh, xp, _dev(np.zeros(c.xyz.shape[0], np.int32)),
                                   batch=0, steps=1)
        assert e.value.code == -1
    finally:
        fresh.close()
