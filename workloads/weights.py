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
