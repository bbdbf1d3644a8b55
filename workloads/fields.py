"""Analytic velocity fields sampled at points (inputs only).

Each function maps points p[n, d] (float64) to velocities u[n, d] (float64).
They stand in for the flow fields the paper's L-G solver would provide
(Sec. 3): solid-body rotation, Taylor-Green and ABC flows, and random
superpositions of Fourier modes for training data.
"""

import numpy as np


def rotation(p, centre=(0.5, 0.5)):
    """Solid-body rotation u = (-(y - cy), x - cx)."""
    u = np.empty_like(p)
    u[:, 0] = -(p[:, 1] - centre[1])
    u[:, 1] = p[:, 0] - centre[0]
    return u


def taylor_green(p):
    """u = (sin(pi x) cos(pi y), -cos(pi x) sin(pi y))."""
    x, y = p[:, 0], p[:, 1]
    u = np.empty_like(p)
    u[:, 0] = np.sin(np.pi * x) * np.cos(np.pi * y)
    u[:, 1] = -np.cos(np.pi * x) * np.sin(np.pi * y)
    return u


def abc_flow(p, A=1.0, B=1.0, C=1.0):
    """Arnold-Beltrami-Childress flow, one period across the unit cube."""
    x, y, z = (2.0 * np.pi * p[:, k] for k in range(3))
    u = np.empty_like(p)
    u[:, 0] = A * np.sin(z) + C * np.cos(y)
    u[:, 1] = B * np.sin(x) + A * np.cos(z)
    u[:, 2] = C * np.sin(y) + B * np.cos(x)
    return u


def _modes(rng, n_modes, dim):
    a = rng.standard_normal((n_modes, dim if dim == 3 else 1))
    k = rng.integers(1, 5, size=(n_modes, 3))
    return a, k


def fourier_modes_2d(p, seed, n_modes=8):
    """Divergence-free 2-D field from a random stream function.

    psi = sum_k a_k sin(pi m_k x) sin(pi n_k y) / pi with a_k ~ N(0,1) and
    m_k, n_k uniform in {1..4}; u = (d psi/dy, -d psi/dx).
    """
    rng = np.random.default_rng(seed)
    a, k = _modes(rng, n_modes, 2)
    x, y = p[:, 0], p[:, 1]
    u = np.zeros_like(p)
    for j in range(n_modes):
        m, n = k[j, 0], k[j, 1]
        u[:, 0] += a[j, 0] * n * np.sin(np.pi * m * x) * np.cos(np.pi * n * y)
        u[:, 1] -= a[j, 0] * m * np.cos(np.pi * m * x) * np.sin(np.pi * n * y)
    return u


def fourier_modes_3d(p, seed, n_modes=8):
    """Divergence-free 3-D field u = curl A from a random vector potential.

    A_c = sum_k a_kc sin(pi m x) sin(pi n y) sin(pi q z) / pi per component c.
    """
    rng = np.random.default_rng(seed)
    a, k = _modes(rng, n_modes, 3)
    x, y, z = p[:, 0], p[:, 1], p[:, 2]
    u = np.zeros_like(p)
    for j in range(n_modes):
        m, n, q = k[j]
        sx, cx = np.sin(np.pi * m * x), np.cos(np.pi * m * x)
        sy, cy = np.sin(np.pi * n * y), np.cos(np.pi * n * y)
        sz, cz = np.sin(np.pi * q * z), np.cos(np.pi * q * z)
        # partial derivatives of phi = sx*sy*sz/pi
        dx, dy, dz = m * cx * sy * sz, n * sx * cy * sz, q * sx * sy * cz
        a1, a2, a3 = a[j]
        u[:, 0] += a3 * dy - a2 * dz
        u[:, 1] += a1 * dz - a3 * dx
        u[:, 2] += a2 * dx - a1 * dy
    return u


def cfl_of(u, dt, h):
    """CFL = max over nodes of |u| dt / h."""
    return float(np.sqrt((u * u).sum(axis=1)).max() * dt / h)


def dt_for_cfl(u, h, cfl):
    """Time step that gives max|u| dt / h = cfl."""
    umax = float(np.sqrt((u * u).sum(axis=1)).max())
    return cfl * h / umax
