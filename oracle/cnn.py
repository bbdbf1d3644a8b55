"""FP64 reference of the CNN start predictor (test infrastructure only).

The paper's predictor (Sec. 2.3, Eq. 7-8) seeds the walk: its output replaces
the particle's own element K_m as the origin of Algorithm 1. This is the
regressor form: a velocity window around the particle goes through valid
3x3 (3x3x3) convolutions with ReLU between layers (Sec. 2.3 uses ReLU between
layers), then two fully connected layers (hidden width h1 = 256, Sec. 3.1),
and the output is the displacement of the particle in ASG cell units.

  2-D: input [2, 9, 9]    -> 4 x conv3x3 (32 ch) -> [32, 1, 1] -> 256 -> 2
  3-D: input [3, 7, 7, 7] -> 3 x conv3^3 (32 ch) -> [32, 1, 1, 1] -> 256 -> 3

Weights are a flat float32 vector in the order below (the library's
predictor buffer uses the same layout); every function here is plain numpy
in float64, one sample at a time or batched with explicit loops over taps.

Layout, for each conv layer l: W_l[C_out=32][C_in][taps] then b_l[32], where
tap t = (dz*3 +) dy*3 + dx and offsets d* in {0,1,2} read input position
(z+dz, y+dy, x+dx) for output position (z, y, x) (cross-correlation). Then
fc1: W[256][32], b[256]; fc2: W[dim][256], b[dim].

Training loss: mean squared error over batch and components,
L = 1/(B*dim) sum (d_hat - d)^2. Optimiser: Adam (Sec. 2.3) with
beta1 = 0.9, beta2 = 0.999, eps = 1e-8.
"""

import numpy as np

CH = 32
HIDDEN = 256


def spec(dim):
    """Layer list [(kind, shape_W, shape_b)] for dim 2 or 3."""
    if dim == 2:
        cin, n_conv, taps = 2, 4, 9
    else:
        cin, n_conv, taps = 3, 3, 27
    layers = []
    c = cin
    for _ in range(n_conv):
        layers.append(("conv", (CH, c, taps), (CH,)))
        c = CH
    layers.append(("fc", (HIDDEN, CH), (HIDDEN,)))
    layers.append(("fc", (dim, HIDDEN), (dim,)))
    return layers


def patch_size(dim):
    return 9 if dim == 2 else 7


def n_params(dim):
    return sum(int(np.prod(w)) + int(np.prod(b)) for _, w, b in spec(dim))


def unpack(dim, flat):
    """Flat vector -> list of (W, b) float64 arrays."""
    flat = np.asarray(flat, dtype=np.float64)
    out, o = [], 0
    for _, ws, bs in spec(dim):
        nw, nb = int(np.prod(ws)), int(np.prod(bs))
        out.append((flat[o:o + nw].reshape(ws), flat[o + nw:o + nw + nb].reshape(bs)))
        o += nw + nb
    assert o == flat.size, (o, flat.size)
    return out


def pack(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def _offsets(dim):
    if dim == 2:
        return [(dy, dx) for dy in range(3) for dx in range(3)]
    return [(dz, dy, dx) for dz in range(3) for dy in range(3) for dx in range(3)]


def conv_valid(x, W, b):
    """x [B, C_in, *S], W [C_out, C_in, taps], b [C_out] -> [B, C_out, *(S-2)]."""
    dim = x.ndim - 2
    S = x.shape[2:]
    So = tuple(s - 2 for s in S)
    out = np.broadcast_to(b.reshape((1, -1) + (1,) * dim), (x.shape[0], W.shape[0]) + So).copy()
    for t, off in enumerate(_offsets(dim)):
        sl = tuple(slice(o, o + so) for o, so in zip(off, So))
        xs = x[(slice(None), slice(None)) + sl]                 # [B, C_in, *So]
        out += np.einsum("oi,bi...->bo...", W[:, :, t], xs)
    return out


def conv_valid_backward(x, W, gout):
    """Gradients of conv_valid: returns (gx, gW, gb)."""
    dim = x.ndim - 2
    So = gout.shape[2:]
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t, off in enumerate(_offsets(dim)):
        sl = tuple(slice(o, o + so) for o, so in zip(off, So))
        xs = x[(slice(None), slice(None)) + sl]
        gW[:, :, t] = np.einsum("bop,bip->oi", gout.reshape(gout.shape[0], gout.shape[1], -1),
                                xs.reshape(xs.shape[0], xs.shape[1], -1))
        gx[(slice(None), slice(None)) + sl] += np.einsum("oi,bo...->bi...", W[:, :, t], gout)
    gb = gout.sum(axis=tuple(i for i in range(gout.ndim) if i != 1))
    return gx, gW, gb


def relu(x):
    return np.maximum(x, 0.0)


def forward(dim, params, patches, keep=False):
    """patches [B, C_in, *S] (float64) -> d_hat [B, dim]; keep=True also returns
    the per-layer inputs and pre-activations needed by backward()."""
    x = np.asarray(patches, dtype=np.float64)
    acts = []
    L = spec(dim)
    for li, ((kind, _, _), (W, b)) in enumerate(zip(L, params)):
        acts.append(x)
        if kind == "conv":
            z = conv_valid(x, W, b)
            x = relu(z)
            if li == sum(1 for k, _, _ in L if k == "conv") - 1:
                x = x.reshape(x.shape[0], -1)
        else:
            z = x @ W.T + b
            x = relu(z) if li < len(L) - 1 else z
        acts.append(z)
    return (x, acts) if keep else x


def mse(dhat, target):
    d = dhat - target
    return float((d * d).mean())


def backward(dim, params, acts, dhat, target):
    """Gradients of the MSE loss with respect to every (W, b)."""
    L = spec(dim)
    B = dhat.shape[0]
    g = 2.0 * (dhat - target) / (B * dim)
    grads = [None] * len(L)
    n_conv = sum(1 for k, _, _ in L if k == "conv")
    for li in range(len(L) - 1, -1, -1):
        kind = L[li][0]
        W, b = params[li]
        x_in, z = acts[2 * li], acts[2 * li + 1]
        if li < len(L) - 1:
            g = g * (z > 0)                      # ReLU after every layer but the last
        if kind == "fc":
            grads[li] = (g.T @ x_in, g.sum(axis=0))
            g = g @ W
            if li == n_conv:                      # back to the conv feature map shape
                g = g.reshape(z.shape[:0] + acts[2 * (li - 1) + 1].shape)
        else:
            gx, gW, gb = conv_valid_backward(x_in, W, g)
            grads[li] = (gW, gb)
            g = gx
    return grads


class Adam:
    """Adam on a flat parameter vector (float64)."""

    def __init__(self, n, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.m = np.zeros(n)
        self.v = np.zeros(n)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps

    def step(self, w, g):
        self.t += 1
        self.m = self.b1 * self.m + (1.0 - self.b1) * g
        self.v = self.b2 * self.v + (1.0 - self.b2) * g * g
        mhat = self.m / (1.0 - self.b1 ** self.t)
        vhat = self.v / (1.0 - self.b2 ** self.t)
        return w - self.lr * mhat / (np.sqrt(vhat) + self.eps)


def windows(U, cells, dim, scale):
    """Input windows around ASG cells: U [*G, dim] grid velocity (x fastest in
    the flat cell index), cells [B] flat cell ids -> [B, dim, *S] of
    U * scale, zero outside the grid (the padding of Sec. 2.3)."""
    U = np.asarray(U, dtype=np.float64)
    G = U.shape[:-1]                             # (Gy, Gx) or (Gz, Gy, Gx)
    S = patch_size(dim)
    r = S // 2
    B = len(cells)
    # channel k (velocity component k) is scaled by scale[k]
    sc = np.broadcast_to(np.asarray(scale, dtype=np.float64), (dim,)).reshape((dim,) + (1,) * dim)
    out = np.zeros((B, dim) + (S,) * dim)
    idx = np.unravel_index(np.asarray(cells), G)  # (iy, ix) or (iz, iy, ix)
    for b in range(B):
        c = [int(i[b]) for i in idx]
        lo = [ci - r for ci in c]
        src = tuple(slice(max(l, 0), min(l + S, g)) for l, g in zip(lo, G))
        dst = tuple(slice(s.start - l, s.stop - l) for s, l in zip(src, lo))
        out[(b, slice(None)) + dst] = np.moveaxis(U[src], -1, 0) * sc
    return out
