"""Pins of the classifier oracle (oracle/classifier.py, Sec. 2.3, Eq. 7-8).

Each check uses arithmetic of its own, not the oracle's routines:
- average pooling and the input window against loops over every element and
  cell, with cells from floor((x - lo) / s) in numpy;
- padding: cells outside the grid carry their own centre;
- the whole forward pass for one sample with every sum written out;
- softmax and cross-entropy identities;
- every layer's gradient against central finite differences (FP64);
- the label cell holds K_t's centroid, and a walk from the seed of that cell
  (the start a perfect classifier gives) ends in the same host;
- a few Adam steps lower the loss.
"""

import numpy as np
import pytest

import oracle
from oracle import classifier as C
from oracle import cnn
from workloads import make_case


@pytest.fixture(scope="module")
def mesh2():
    c = make_case("rotation2d", n_side=21)
    return c, oracle.Mesh(c.xyz, c.conn)


@pytest.fixture(scope="module")
def mesh3():
    c = make_case("abc3d", n_side=6, cfl=2)
    return c, oracle.Mesh(c.xyz, c.conn)


def _cell_xyz(om, pts):
    s = (om.hi - om.lo) / om.grid
    return np.clip(np.floor((pts - om.lo) / s).astype(np.int64), 0, om.grid - 1)


def test_pooling_is_the_mean_centroid_per_cell(mesh2, mesh3):
    for c, om in (mesh2, mesh3):
        mean, cnt = C.pooled_cells(om)
        cen = c.xyz[c.conn].sum(axis=1) / (c.dim + 1)
        cc = _cell_xyz(om, cen)
        g = om.grid
        want_sum = {}
        for e in range(c.n_elements):
            key = tuple(cc[e])
            want_sum.setdefault(key, []).append(cen[e])
        for idx in np.ndindex(*[int(v) for v in g[::-1]]):
            key = tuple(idx[::-1])
            flat = 0
            for k in range(c.dim - 1, -1, -1):
                flat = flat * int(g[k]) + key[k]
            pts = want_sum.get(key, [])
            assert cnt[flat] == len(pts)
            if pts:
                assert np.allclose(mean[flat], np.mean(pts, axis=0), rtol=0, atol=1e-15)


def test_window_features_by_explicit_loops(mesh2):
    c, om = mesh2
    W = C.window_size(2)
    s = (om.hi - om.lo) / om.grid
    cen = c.xyz[c.conn].mean(axis=1)
    cc = _cell_xyz(om, cen)
    rng = np.random.default_rng(4)
    xp = np.concatenate([rng.random((6, 2)), [[0.01, 0.02], [0.995, 0.5]]])
    win, off, _ = C.features(om, xp)
    for b in range(xp.shape[0]):
        ic = _cell_xyz(om, xp[b:b + 1])[0]
        assert np.allclose(off[b], (xp[b] - om.lo) / s - (ic + 0.5), atol=1e-13)
        for wy in range(W):
            for wx in range(W):
                cell = ic + np.array([wx, wy]) - W // 2
                members = [cen[e] for e in range(c.n_elements) if (cc[e] == cell).all()]
                inside = (cell >= 0).all() and (cell < om.grid).all()
                pt = np.mean(members, axis=0) if (inside and members) else om.lo + (cell + 0.5) * s
                assert np.allclose(win[b, :, wy, wx], (pt - xp[b]) / s, atol=1e-12), (b, wy, wx)


def test_softmax_and_cross_entropy(mesh2):
    c, om = mesh2
    xp = c.x[:16] - c.u[:16] * c.dt
    win, off, _ = C.features(om, xp)
    params = C.init(2, 1)
    H, P = C.forward(params, win, off)
    assert np.allclose(P.sum(axis=1), 1.0, atol=1e-14)
    assert np.allclose(C.softmax(H + 123.0), P, atol=1e-15)
    lab = np.arange(16) % H.shape[1]
    manual = -np.mean([H[i, lab[i]] - np.log(np.exp(H[i]).sum()) for i in range(16)])
    assert abs(C.cross_entropy(P, lab) - manual) < 1e-12


@pytest.mark.parametrize("dim,W", [(2, 5), (3, 3)])
def test_gradients_match_finite_differences(mesh2, mesh3, dim, W):
    c, om = mesh2 if dim == 2 else mesh3
    rng = np.random.default_rng(7)
    xp = c.x[:3] - c.u[:3] * c.dt
    win, off, _ = C.features(om, xp, W=W)
    win = win + 0.3 * rng.standard_normal(win.shape)       # exercise every ReLU branch
    params = C.init(dim, 2, W=W)
    params = [(w + 0.05 * rng.standard_normal(w.shape), b + 0.05 * rng.standard_normal(b.shape))
              for w, b in params]
    lab = rng.integers(0, W ** dim, size=3)
    _, P, keep = C.forward(params, win, off, keep=True)
    grads = C.backward(params, P, lab, keep)
    h = 1e-6
    for li, ((w, b), (gw, gb)) in enumerate(zip(params, grads)):
        for arr, g in ((w, gw), (b, gb)):
            flat = arr.reshape(-1)
            for j in rng.choice(flat.size, size=min(6, flat.size), replace=False):
                old = flat[j]
                flat[j] = old + h
                lp = C.cross_entropy(C.forward(params, win, off)[1], lab)
                flat[j] = old - h
                lm = C.cross_entropy(C.forward(params, win, off)[1], lab)
                flat[j] = old
                fd = (lp - lm) / (2 * h)
                assert abs(fd - g.reshape(-1)[j]) <= 1e-6 + 1e-5 * abs(fd), (li, j, fd)


def test_labels_and_the_perfect_classifier_start(mesh2):
    c, om = mesh2
    xp = c.x - c.u * c.dt
    r = om.track(c.x, c.u, c.dt)
    found = r["host"] >= 0
    lab = C.labels(om, xp[found], r["host"][found])
    W = C.window_size(2)
    # the label's cell holds the host's centroid (none is clamped here)
    cen = c.xyz[c.conn[r["host"][found]]].mean(axis=1)
    ic = _cell_xyz(om, xp[found])
    rel = _cell_xyz(om, cen) - ic + W // 2
    assert ((rel >= 0) & (rel < W)).all()
    assert np.array_equal(lab, rel[:, 1] * W + rel[:, 0])
    # K_p = seed of that cell; walking from it gives the same hosts
    kp = C.start_elements(om, xp[found], lab)
    assert (kp >= 0).all()
    r2 = om.track(c.x[found], c.u[found], c.dt, start=kp)
    assert np.array_equal(r2["host"], r["host"][found])
    assert r2["path_len"].mean() < r["path_len"][found].mean()


def test_a_sample_without_host_has_no_label(mesh2):
    """A departure point outside the mesh has host -1 (R8) and so no K_t:
    its label is -1, and the labels of the other samples do not change."""
    c, om = mesh2
    xp = np.array([[0.5, 0.5], [2.0, 0.5], [0.25, 0.75]])
    host = om.locate(xp)
    assert host[1] == -1 and host[0] >= 0 and host[2] >= 0
    lab = C.labels(om, xp, host)
    assert lab[1] == -1
    assert np.array_equal(lab[[0, 2]], C.labels(om, xp[[0, 2]], host[[0, 2]]))


def test_adam_steps_lower_the_loss(mesh2):
    c, om = mesh2
    xp = c.x - c.u * c.dt
    r = om.track(c.x, c.u, c.dt)
    ok = np.nonzero(r["host"] >= 0)[0][:128]
    win, off, _ = C.features(om, xp[ok])
    lab = C.labels(om, xp[ok], r["host"][ok])
    params = C.init(2, 3)
    shapes = [(w.shape, b.shape) for w, b in params]
    flat = np.concatenate([np.concatenate([w.reshape(-1), b]) for w, b in params])
    opt = cnn.Adam(flat.size, lr=1e-3)

    def unflat(v):
        out, o = [], 0
        for ws, bs in shapes:
            nw, nb = int(np.prod(ws)), int(np.prod(bs))
            out.append((v[o:o + nw].reshape(ws), v[o + nw:o + nw + nb]))
            o += nw + nb
        return out

    losses = []
    for _ in range(30):
        p = unflat(flat)
        _, P, keep = C.forward(p, win, off, keep=True)
        losses.append(C.cross_entropy(P, lab))
        g = C.backward(p, P, lab, keep)
        gflat = np.concatenate([np.concatenate([gw.reshape(-1), gb]) for gw, gb in g])
        flat = opt.step(flat, gflat)
    assert losses[-1] < 0.5 * losses[0], (losses[0], losses[-1])


def test_forward_by_explicit_loops(mesh2):
    """One sample through the whole network, every sum written out: zero-
    padded 3x3 cross-correlations (tap (dy, dx) reads (y + dy - 1, x + dx - 1)),
    ReLU, 2x2 average pooling from the window's first row and column, the x_p
    branch, the fusion layer and the logits."""
    c, om = mesh2
    W = 5
    rng = np.random.default_rng(11)
    xp = c.x[7:8] - c.u[7:8] * c.dt
    win, off, _ = C.features(om, xp, W=W)
    params = [(w + 0.1 * rng.standard_normal(w.shape), b + 0.1 * rng.standard_normal(b.shape))
              for w, b in C.init(2, 5, W=W)]
    (W1, b1), (W2, b2), (X1, c1), (X2, c2), (F, f), (L, l) = params
    relu = lambda v: max(v, 0.0)

    def conv(x, Wt, b):
        cout, cin = Wt.shape[0], Wt.shape[1]
        out = np.zeros((cout, W, W))
        for o in range(cout):
            for y in range(W):
                for xx in range(W):
                    acc = b[o]
                    for i in range(cin):
                        for dy in range(3):
                            for dx in range(3):
                                yy, xs = y + dy - 1, xx + dx - 1
                                if 0 <= yy < W and 0 <= xs < W:
                                    acc += Wt[o, i, dy * 3 + dx] * x[i, yy, xs]
                    out[o, y, xx] = relu(acc)
        return out

    a1 = conv(win[0], W1, b1)
    a2 = conv(a1, W2, b2)
    Wp = W // 2
    pooled = np.zeros((C.CH, Wp, Wp))
    for o in range(C.CH):
        for y in range(Wp):
            for xx in range(Wp):
                pooled[o, y, xx] = (a2[o, 2 * y, 2 * xx] + a2[o, 2 * y, 2 * xx + 1] +
                                    a2[o, 2 * y + 1, 2 * xx] + a2[o, 2 * y + 1, 2 * xx + 1]) / 4
    y1 = [relu(c1[j] + sum(X1[j, k] * off[0, k] for k in range(2))) for j in range(C.H1)]
    y2 = [relu(c2[j] + sum(X2[j, k] * y1[k] for k in range(C.H1))) for j in range(C.H1)]
    cat = list(pooled.reshape(-1)) + y2
    u = [relu(f[j] + sum(F[j, k] * cat[k] for k in range(len(cat)))) for j in range(C.H2)]
    H = np.array([l[j] + sum(L[j, k] * u[k] for k in range(C.H2)) for j in range(W * W)])
    got, _ = C.forward(params, win, off)
    assert np.allclose(got[0], H, rtol=1e-12, atol=1e-10)
