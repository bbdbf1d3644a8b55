"""Reported metrics of the paper, written out plainly (test infrastructure).

err (Sec. 3.1): distance between the centroid of the tracking origin and the
centroid of the host K_t; the origin is K_m for SNS and K_p for CNN-SNS.
Opt(C) (Sec. 3.1): (C(SNS) - C(CNN-SNS)) / C(SNS).
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
