"""FP64 reference of the paper's classifier predictor (Sec. 2.3, Eq. 7-8).

Test infrastructure only: only tests/, the smoke check and bench.py's CPU
baseline leg may import it; the product path never does.

The paper's CNN classifies x_p among the elements of a filtered window around
it. Its input is the element centroids (Sec. 2.3: x_l* = mean of the element's
vertices) of the elements in a cubic ASG-grid region around x_p, averaged per
grid cell (average pooling) and padded at the domain boundary, plus x_p
itself. Two modules read them: two convolutions and a pooling layer on the
centroids, two fully connected layers on x_p. The two outputs are
concatenated and go through two fully connected layers to logits, then a
softmax over the window (B_l, Eq. 7). The most probable class gives K_p
(Eq. 8). The label is one-hot on the class of K_t found by SNS, and the loss
is the cross-entropy. ReLU runs between layers.

Where the text leaves the shape open, this module reads it as follows (one
reading each, listed with the others):
- window: W^d ASG cells (W odd) centred on the cell of x_p, so x_p always
  lies inside it; the classes are those W^d cells (N_a = W^d);
- cell features: the mean centroid of the elements whose centroid lies in
  the cell, minus x_p, in ASG cell units; a cell outside the grid or without
  an element centroid is padded with its own centre;
- module 1: conv 3^d (d -> 32 channels) and conv 3^d (32 -> 32), zero
  padded to keep the window size, ReLU after each, then average pooling over
  2^d blocks (stride 2, the last odd row dropped);
- module 2: x_p's offset from its cell's centre, in cell units, through two
  fully connected layers of width h1 = 256 (Sec. 3.1), ReLU after each;
- fusion: concatenation, a fully connected layer of width h2 = 512 (Sec.
  3.1) with ReLU, and one to the W^d logits;
- the label is the window cell that holds K_t's centroid (clamped into the
  window); K_p is the ASG seed of the predicted cell, the element that
  contains the cell's centre.

Weights are a list of (W, b) float64 arrays; conv W is [C_out][C_in][taps]
with the tap order of oracle.cnn.
"""

import numpy as np

from . import cnn as _cnn
from . import grid_cells

CH = 32
H1 = 256
H2 = 512


def window_size(dim):
    """W: 9 cells per axis in 2-D (81 classes), 7 in 3-D (343)."""
    return 9 if dim == 2 else 7


def spec(dim, W=None):
    """[(name, shape_W, shape_b)] of the classifier for dim 2 or 3."""
    W = W or window_size(dim)
    taps = 3 ** dim
    pooled = CH * (W // 2) ** dim
    n_cls = W ** dim
    return [("conv1", (CH, dim, taps), (CH,)),
            ("conv2", (CH, CH, taps), (CH,)),
            ("xp1", (H1, dim), (H1,)),
            ("xp2", (H1, H1), (H1,)),
            ("fuse", (H2, pooled + H1), (H2,)),
            ("logits", (n_cls, H2), (n_cls,))]


def init(dim, seed, W=None):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    params = []
    for _, ws, bs in spec(dim, W):
        fan_in = int(np.prod(ws[1:]))
        params.append((rng.standard_normal(ws) * np.sqrt(2.0 / fan_in), np.zeros(bs)))
    return params


def cell_coords(om, cells):
    """Flat ASG cell index (x fastest) -> integer coordinates [n, dim]."""
    g = om.grid.astype(np.int64)
    out = np.empty((len(cells), om.dim), dtype=np.int64)
    r = np.asarray(cells, dtype=np.int64)
    for k in range(om.dim):
        out[:, k] = r % g[k]
        r = r // g[k]
    return out


def pooled_cells(om):
    """Average pooling over the whole grid: per ASG cell the mean centroid of
    the elements whose centroid lies in it, and the count (0: empty)."""
    cen = om.centroids()
    c = grid_cells(om.lo, om.hi, om.grid, cen)
    n = int(np.prod(om.grid.astype(np.int64)))
    cnt = np.bincount(c, minlength=n)
    acc = np.zeros((n, om.dim))
    for k in range(om.dim):
        acc[:, k] = np.bincount(c, weights=cen[:, k], minlength=n)
    mean = np.where(cnt[:, None] > 0, acc / np.maximum(cnt, 1)[:, None], np.nan)
    return mean, cnt


def features(om, xp, W=None, pooled=None):
    """Inputs of the two modules for departure points xp [B, dim]:
    window [B, dim, W, ..., W] (z, y, x order of the spatial axes, x fastest)
    and offset [B, dim]; also the window's first cell coordinates [B, dim]."""
    dim = om.dim
    W = W or window_size(dim)
    mean, cnt = pooled if pooled is not None else pooled_cells(om)
    xp = np.asarray(xp, dtype=np.float64)
    s = (om.hi - om.lo) / om.grid
    centre_cell = cell_coords(om, grid_cells(om.lo, om.hi, om.grid, xp))
    first = centre_cell - W // 2
    B = xp.shape[0]
    win = np.empty((B, dim) + (W,) * dim)
    g = om.grid.astype(np.int64)
    for idx in np.ndindex(*((W,) * dim)):            # (z,) y, x window offsets
        off = np.array(idx[::-1])                     # x first
        cc = first + off                              # [B, dim] integer cell coords
        inside = np.all((cc >= 0) & (cc < g), axis=1)
        flat = np.zeros(B, dtype=np.int64)
        for k in range(dim - 1, -1, -1):
            flat = flat * g[k] + np.clip(cc[:, k], 0, g[k] - 1)
        has = inside & (cnt[flat] > 0)
        pt = np.where(has[:, None], mean[flat], om.lo + (cc + 0.5) * s)
        win[(slice(None), slice(None)) + idx] = (pt - xp) / s
    offset = (xp - om.lo) / s - (centre_cell + 0.5)
    return win, offset, first


def _pool(x):
    """Average pooling over 2^d blocks, stride 2, odd remainder dropped."""
    dim = x.ndim - 2
    Wp = x.shape[2] // 2
    out = np.zeros(x.shape[:2] + (Wp,) * dim)
    for off in np.ndindex(*((2,) * dim)):
        sl = tuple(slice(o, o + 2 * Wp, 2) for o in off)
        out += x[(slice(None), slice(None)) + sl]
    return out / (2 ** dim)


def _pool_backward(g, shape):
    dim = g.ndim - 2
    Wp = g.shape[2]
    gx = np.zeros(shape)
    for off in np.ndindex(*((2,) * dim)):
        sl = tuple(slice(o, o + 2 * Wp, 2) for o in off)
        gx[(slice(None), slice(None)) + sl] += g / (2 ** dim)
    return gx


def _pad1(x):
    dim = x.ndim - 2
    return np.pad(x, [(0, 0), (0, 0)] + [(1, 1)] * dim)


def softmax(h):
    z = h - h.max(axis=1, keepdims=True)
    e = np.exp(z)
    return e / e.sum(axis=1, keepdims=True)


def forward(params, win, offset, keep=False):
    """Logits H [B, W^d] and probabilities B_l (Eq. 7); keep=True also
    returns the intermediate values backward() needs."""
    (W1, b1), (W2, b2), (X1, c1), (X2, c2), (F, f), (L, l) = params
    a0 = _pad1(win)
    z1 = _cnn.conv_valid(a0, W1, b1)
    a1 = _pad1(_cnn.relu(z1))
    z2 = _cnn.conv_valid(a1, W2, b2)
    p = _pool(_cnn.relu(z2))
    y1 = offset @ X1.T + c1
    y2 = _cnn.relu(y1) @ X2.T + c2
    cat = np.concatenate([p.reshape(p.shape[0], -1), _cnn.relu(y2)], axis=1)
    u = cat @ F.T + f
    H = _cnn.relu(u) @ L.T + l
    P = softmax(H)
    if keep:
        return H, P, dict(a0=a0, z1=z1, a1=a1, z2=z2, p=p, y1=y1, y2=y2, cat=cat, u=u,
                          offset=offset)
    return H, P


def cross_entropy(P, labels):
    """Mean over the batch of -log B_t (the loss of Sec. 2.3 with one-hot B')."""
    return float(-np.log(P[np.arange(P.shape[0]), labels]).mean())


def backward(params, P, labels, keep):
    """Gradients of cross_entropy with respect to every (W, b)."""
    (W1, b1), (W2, b2), (X1, c1), (X2, c2), (F, f), (L, l) = params
    Bn = P.shape[0]
    gH = P.copy()
    gH[np.arange(Bn), labels] -= 1.0
    gH /= Bn                                              # d CE / d logits
    gL = gH.T @ _cnn.relu(keep["u"])
    gl = gH.sum(axis=0)
    gu = (gH @ L) * (keep["u"] > 0)
    gF = gu.T @ keep["cat"]
    gf = gu.sum(axis=0)
    gcat = gu @ F
    n_pool = keep["p"][0].size
    gp = gcat[:, :n_pool].reshape(keep["p"].shape)
    gy2 = gcat[:, n_pool:] * (keep["y2"] > 0)
    gX2 = gy2.T @ _cnn.relu(keep["y1"])
    gc2 = gy2.sum(axis=0)
    gy1 = (gy2 @ X2) * (keep["y1"] > 0)
    gX1 = gy1.T @ keep["offset"]
    gc1 = gy1.sum(axis=0)
    gz2 = _pool_backward(gp, keep["z2"].shape) * (keep["z2"] > 0)
    ga1, gW2, gb2 = _cnn.conv_valid_backward(keep["a1"], W2, gz2)
    core = tuple(slice(1, -1) for _ in range(ga1.ndim - 2))
    gz1 = ga1[(slice(None), slice(None)) + core] * (keep["z1"] > 0)
    _, gW1, gb1 = _cnn.conv_valid_backward(keep["a0"], W1, gz1)
    return [(gW1, gb1), (gW2, gb2), (gX1, gc1), (gX2, gc2), (gF, gf), (gL, gl)]


def labels(om, xp, host, W=None):
    """Class of each sample: the window cell that holds the centroid of its
    host K_t (user ids), clamped into the window around xp; -1 where the
    sample has no host (host -1: x_p outside the mesh, so there is no K_t)."""
    W = W or window_size(om.dim)
    host = np.asarray(host)
    cen = om.centroids()[np.maximum(host, 0)]
    centre_cell = cell_coords(om, grid_cells(om.lo, om.hi, om.grid, xp))
    first = centre_cell - W // 2
    cc = cell_coords(om, grid_cells(om.lo, om.hi, om.grid, cen))
    rel = np.clip(cc - first, 0, W - 1)
    cls = np.zeros(len(xp), dtype=np.int64)
    for k in range(om.dim - 1, -1, -1):
        cls = cls * W + rel[:, k]
    return np.where(host >= 0, cls, -1)


def start_elements(om, xp, cls, W=None):
    """K_p (Eq. 8): the ASG seed of the predicted window cell (user id, or -1
    where the cell lies outside the grid or its centre outside the mesh)."""
    W = W or window_size(om.dim)
    centre_cell = cell_coords(om, grid_cells(om.lo, om.hi, om.grid, xp))
    first = centre_cell - W // 2
    rel = np.zeros((len(cls), om.dim), dtype=np.int64)
    r = np.asarray(cls, dtype=np.int64)
    for k in range(om.dim):
        rel[:, k] = r % W
        r = r // W
    cc = first + rel
    g = om.grid.astype(np.int64)
    inside = np.all((cc >= 0) & (cc < g), axis=1)
    flat = np.zeros(len(cls), dtype=np.int64)
    for k in range(om.dim - 1, -1, -1):
        flat = flat * g[k] + np.clip(cc[:, k], 0, g[k] - 1)
    return np.where(inside, om.seed[flat], -1).astype(np.int32)
