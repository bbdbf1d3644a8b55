"""Pins for the oracle's CNN start predictor (CPU only): finite differences,
an independent correlation routine, a hand-built network with a closed-form
output, the closed form of Adam's first step, and the window geometry."""

import numpy as np
import pytest

from oracle import cnn
from workloads.weights import init_weights, layer_shapes


@pytest.mark.parametrize("dim", [2, 3])
def test_layout_matches_generator(dim):
    assert [(w, b) for _, w, b in cnn.spec(dim)] == layer_shapes(dim)
    assert cnn.n_params(dim) == (37314 if dim == 2 else 67203)
    flat = init_weights(dim, 1)
    assert flat.size == cnn.n_params(dim)
    assert np.array_equal(cnn.pack(cnn.unpack(dim, flat)), flat.astype(np.float64))


@pytest.mark.parametrize("dim", [2, 3])
def test_conv_matches_scipy_correlate(dim):
    from scipy.signal import correlate
    rng = np.random.default_rng(2)
    S = 6
    x = rng.standard_normal((2, 3) + (S,) * dim)
    W = rng.standard_normal((4, 3, 3 ** dim))
    b = rng.standard_normal(4)
    out = cnn.conv_valid(x, W, b)
    for bi in range(2):
        for o in range(4):
            ref = b[o] + sum(correlate(x[bi, i], W[o, i].reshape((3,) * dim), mode="valid")
                             for i in range(3))
            assert np.allclose(out[bi, o], ref, atol=1e-12)


@pytest.mark.parametrize("dim", [2, 3])
def test_backward_matches_finite_differences(dim):
    rng = np.random.default_rng(5)
    flat = init_weights(dim, 3).astype(np.float64)
    flat += 0.05 * rng.standard_normal(flat.size)       # non-zero biases too
    S = cnn.patch_size(dim)
    x = rng.standard_normal((3, dim) + (S,) * dim)
    t = rng.standard_normal((3, dim))
    params = cnn.unpack(dim, flat)
    dhat, acts = cnn.forward(dim, params, x, keep=True)
    g = cnn.pack(cnn.backward(dim, params, acts, dhat, t))

    def loss(w):
        return cnn.mse(cnn.forward(dim, cnn.unpack(dim, w), x), t)

    idx = rng.choice(flat.size, size=60, replace=False)
    h = 1e-6
    for i in idx:
        wp, wm = flat.copy(), flat.copy()
        wp[i] += h
        wm[i] -= h
        fd = (loss(wp) - loss(wm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def _passthrough_weights(dim):
    """Conv layers copy +u_k and -u_k of the centre into 2*dim channels
    (ReLU keeps each sign apart), fc1 passes them on, fc2 forms
    -(pos - neg) = -u_k: the network outputs minus the centre pixel."""
    params = []
    for ws, bs in layer_shapes(dim):
        params.append([np.zeros(ws), np.zeros(bs)])
    centre = 4 if dim == 2 else 13
    n_conv = 4 if dim == 2 else 3
    for l in range(n_conv):
        W = params[l][0]
        for k in range(dim):
            if l == 0:
                W[2 * k, k, centre] = 1.0
                W[2 * k + 1, k, centre] = -1.0
            else:
                W[2 * k, 2 * k, centre] = 1.0
                W[2 * k + 1, 2 * k + 1, centre] = 1.0
    W1 = params[n_conv][0]
    for c in range(2 * dim):
        W1[c, c] = 1.0
    W2 = params[n_conv + 1][0]
    for k in range(dim):
        W2[k, 2 * k] = -1.0
        W2[k, 2 * k + 1] = 1.0
    return [(W, b) for W, b in params]


@pytest.mark.parametrize("dim", [2, 3])
def test_handbuilt_network_outputs_minus_centre(dim):
    """With R7 the true displacement is -u(x) dt, i.e. minus the centre pixel
    of the window in cell units: this network computes exactly that."""
    rng = np.random.default_rng(7)
    S = cnn.patch_size(dim)
    x = rng.standard_normal((5, dim) + (S,) * dim)
    out = cnn.forward(dim, _passthrough_weights(dim), x)
    c = (slice(None), slice(None)) + (S // 2,) * dim
    assert np.allclose(out, -x[c], atol=1e-14)


def test_adam_first_step_closed_form():
    """After one step m_hat = g and v_hat = g^2, so w1 = w0 - lr g/(|g|+eps)."""
    rng = np.random.default_rng(1)
    w0 = rng.standard_normal(50)
    g = rng.standard_normal(50)
    opt = cnn.Adam(50, lr=1e-3)
    w1 = opt.step(w0, g)
    assert np.allclose(w1, w0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    # second step against the recurrence written out
    g2 = rng.standard_normal(50)
    w2 = opt.step(w1, g2)
    m = 0.9 * (0.1 * g) + 0.1 * g2
    v = 0.999 * (0.001 * g * g) + 0.001 * g2 * g2
    ref = w1 - 1e-3 * (m / (1 - 0.81)) / (np.sqrt(v / (1 - 0.998001)) + 1e-8)
    assert np.allclose(w2, ref, rtol=1e-12, atol=0)


def test_windows_geometry_and_padding():
    Gy, Gx = 6, 11
    iy, ix = np.meshgrid(np.arange(Gy), np.arange(Gx), indexing="ij")
    U = np.stack([ix, iy], axis=-1).astype(np.float64)     # U_x = ix, U_y = iy
    cells = np.array([2 * Gx + 5, 0])                       # (iy=2, ix=5) and the corner
    w = cnn.windows(U, cells, 2, scale=[2.0, 3.0])
    # window row r, column q reads cell (iy - 4 + r, ix - 4 + q)
    for r in range(9):
        for q in range(9):
            yy, xx = 2 - 4 + r, 5 - 4 + q
            inside = 0 <= yy < Gy and 0 <= xx < Gx
            assert w[0, 0, r, q] == (2.0 * xx if inside else 0.0)
            assert w[0, 1, r, q] == (3.0 * yy if inside else 0.0)
    assert w[1, 0, 4, 4] == 0.0 and w[1, 0, 4, 5] == 2.0 and w[1, 0, 3, 4] == 0.0
