"""Seeded initial weights of the start predictor (inputs only).

Flat float32 vector in the predictor layout: for each conv layer W[32][C_in]
[taps] then b[32]; then fc1 W[256][32], b[256]; fc2 W[dim][256], b[dim].
He-normal weights (std sqrt(2 / fan_in)), zero biases.
"""

import numpy as np


def layer_shapes(dim):
    cin, n_conv, taps = (2, 4, 9) if dim == 2 else (3, 3, 27)
    shapes = []
    c = cin
    for _ in range(n_conv):
        shapes.append(((32, c, taps), (32,)))
        c = 32
    shapes.append(((256, 32), (256,)))
    shapes.append(((dim, 256), (dim,)))
    return shapes


def init_weights(dim, seed):
    rng = np.random.default_rng(seed)
    parts = []
    for ws, bs in layer_shapes(dim):
        fan_in = int(np.prod(ws[1:]))
        parts.append(rng.standard_normal(int(np.prod(ws))) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(int(np.prod(bs))))
    return np.concatenate(parts).astype(np.float32)


def classifier_layer_shapes(dim):
    """(W shape, b shape) of the classifier's layers: conv1 [32][dim][taps],
    conv2 [32][32][taps], xp1 [256][dim], xp2 [256][256], fuse [512][32 *
    (W/2)^dim + 256], logits [W^dim][512]; W = 9 (2-D) or 7 (3-D)."""
    W, taps = (9, 9) if dim == 2 else (7, 27)
    pooled = 32 * (W // 2) ** dim
    return [((32, dim, taps), (32,)), ((32, 32, taps), (32,)), ((256, dim), (256,)),
            ((256, 256), (256,)), ((512, pooled + 256), (512,)), ((W ** dim, 512), (W ** dim,))]


def init_classifier(dim, seed):
    """Flat float32 parameters of the classifier (W then b per layer, in the
    order of classifier_layer_shapes): He-normal weights, zero biases."""
    rng = np.random.default_rng(seed)
    parts = []
    for ws, bs in classifier_layer_shapes(dim):
        fan_in = int(np.prod(ws[1:]))
        parts.append(rng.standard_normal(int(np.prod(ws))) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(int(np.prod(bs))))
    return np.concatenate(parts).astype(np.float32)
