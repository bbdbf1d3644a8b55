"""Reported metrics of the paper, written out plainly (test infrastructure).

err (Sec. 3.1): distance between the centroid of the tracking origin and the
centroid of the host K_t; the origin is K_m for SNS and K_p for CNN-SNS.
Opt(C) (Sec. 3.1): (C(SNS) - C(CNN-SNS)) / C(SNS).
Displacement error of the start predictor: |d_hat - d| with d = x_p - x the
true displacement (Sec. 2.1, Eq. 3) and d_hat the prediction in length units.
"""

import numpy as np


def opt(c_sns, c_cnn):
    """Optimisation rate of CNN-SNS over SNS for a cost C (a fraction)."""
    return (c_sns - c_cnn) / c_sns


def centroids(xyz, conn):
    """x_l^* = mean of the element's vertices (Sec. 2.3)."""
    return np.asarray(xyz, dtype=np.float64)[np.asarray(conn)].mean(axis=1)


def err(cent, origin, host):
    """Per-particle origin error; entries with origin or host -1 are NaN."""
    origin = np.asarray(origin)
    host = np.asarray(host)
    ok = (origin >= 0) & (host >= 0)
    out = np.full(origin.shape[0], np.nan)
    d = cent[origin[ok]] - cent[host[ok]]
    out[ok] = np.sqrt((d * d).sum(axis=1))
    return out


def path_stats(path_len):
    p = np.asarray(path_len, dtype=np.int64)
    return dict(mean=float(p.mean()) if p.size else 0.0,
                max=int(p.max()) if p.size else 0,
                total=int(p.sum()))


def displacement_error(dhat_cells, cell_size, x, xp):
    """Per-particle |dhat * s - (x_p - x)|: dhat_cells [n, dim] the prediction
    at each particle's predictor cell in cell units (float32 values),
    cell_size [dim] the predictor cell size; entries with a non-finite x_p are
    NaN."""
    d_hat = np.asarray(dhat_cells, dtype=np.float32).astype(np.float64) * np.asarray(cell_size)
    d = np.asarray(xp, dtype=np.float64) - np.asarray(x, dtype=np.float64)
    e = np.sqrt(((d_hat - d) ** 2).sum(axis=1))
    return np.where(np.isfinite(xp).all(axis=1), e, np.nan)
