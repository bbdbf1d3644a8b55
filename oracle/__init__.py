"""CPU oracle of the CNN-SNS particle-location path.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the product path never does.

The particle-location part is plain C (oracle.c, single-threaded, FP64, user
element ids, no reordering) reached through ctypes; the learned start
predictor is plain numpy in FP64 (cnn.py). Nothing here shares code with the
CUDA library.

Result definition (Sec. 2.2 containment test with tolerance eps): the host of
x_p is the lowest user id l with every lambda_i^l(x_p) >= -eps, or -1.
Algorithm 1 gives the path length I_t from a start element.
"""

import ctypes
import functools

import numpy as np

from . import build as _build

EPS = 1e-12

# walk exits
CONTAINED, BOUNDARY, CAP, INVALID = 0, 1, 2, 3
# track status (same codes as the library)
ST_FOUND, ST_OUTSIDE, ST_FALLBACK, ST_INVALID = 0, 1, 2, 3

_f64 = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_u8 = ctypes.POINTER(ctypes.c_uint8)
_i64t = ctypes.c_int64


@functools.lru_cache(maxsize=1)
def lib():
    path = _build.build()
    L = ctypes.CDLL(path)
    sig = {
        "or_set_threads": (ctypes.c_int, [ctypes.c_int]),
        "or_neighbors": (ctypes.c_int, [ctypes.c_int, _i64t, _i32, _i32]),
        "or_neighbors_bruteforce": (ctypes.c_int, [ctypes.c_int, _i64t, _i32, _i32]),
        "or_inverse_affine": (_i64t, [ctypes.c_int, _f64, _i64t, _i32, _f64, _f64]),
        "or_bary": (None, [ctypes.c_int, _f64, _f64, _f64, _f64]),
        "or_bary_det": (None, [ctypes.c_int, _f64, _f64, _f64]),
        "or_departure": (None, [ctypes.c_int, _i64t, _f64, _f64, ctypes.c_double, _f64]),
        "or_locate_bruteforce": (None, [ctypes.c_int, _i64t, _f64, _f64, _i64t, _f64,
                                        ctypes.c_double, _i32]),
        "or_locate_bucketed": (ctypes.c_int, [ctypes.c_int, _i64t, _f64, _i64t, _i32, _f64,
                                              _f64, _i64t, _f64, ctypes.c_double,
                                              ctypes.c_int, _i32]),
        "or_walk": (None, [ctypes.c_int, _f64, _f64, _i32, _i64t, _f64, _i32,
                           ctypes.c_double, ctypes.c_int32, _i32, _i32, _u8]),
        "or_node_elements": (None, [ctypes.c_int, _i64t, _i64t, _i32, _i32]),
        "or_grid_centres": (None, [ctypes.c_int, _f64, _f64, _i32, _f64]),
        "or_grid_cell": (_i64t, [ctypes.c_int, _f64, _f64, _i32, _f64]),
        "or_grid_cells": (None, [ctypes.c_int, _f64, _f64, _i32, _i64t, _f64,
                                 ctypes.POINTER(ctypes.c_int64)]),
        "or_p1_interpolate": (None, [ctypes.c_int, _i32, _f64, _f64, _f64, _i64t, _f64,
                                     _i32, _f64]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


def set_threads(n):
    """Threads of the walk and exact-location loops (1 by default); returns
    the count in effect (1 when the library has no OpenMP)."""
    return int(lib().or_set_threads(int(n)))


def _p(a, ct):
    return a.ctypes.data_as(ct)


def _f(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ---------------------------------------------------------------------------
# primitives
# ---------------------------------------------------------------------------

def neighbors(dim, conn, brute=False):
    conn = _i(conn)
    nbr = np.empty_like(conn)
    fn = lib().or_neighbors_bruteforce if brute else lib().or_neighbors
    rc = fn(dim, conn.shape[0], _p(conn, _i32), _p(nbr, _i32))
    if rc != 0:
        raise ValueError("non-manifold mesh (a face shared by more than two elements)")
    return nbr


def inverse_affine(xyz, conn):
    xyz, conn = _f(xyz), _i(conn)
    dim = xyz.shape[1]
    n_e = conn.shape[0]
    v0 = np.empty((n_e, dim))
    M = np.empty((n_e, dim, dim))
    bad = lib().or_inverse_affine(dim, _p(xyz, _f64), n_e, _p(conn, _i32),
                                  _p(v0, _f64), _p(M, _f64))
    if bad:
        raise ValueError("degenerate element %d" % (bad - 1))
    return v0, M


def bary(v0, M, p):
    v0, M, p = _f(v0), _f(M), _f(p)
    dim = v0.shape[-1]
    lam = np.empty(dim + 1)
    lib().or_bary(dim, _p(v0, _f64), _p(M, _f64), _p(p, _f64), _p(lam, _f64))
    return lam


def bary_det(verts, p):
    verts, p = _f(verts), _f(p)
    dim = verts.shape[1]
    lam = np.empty(dim + 1)
    lib().or_bary_det(dim, _p(verts, _f64), _p(p, _f64), _p(lam, _f64))
    return lam


def departure(x, u, dt):
    x, u = _f(x), _f(u)
    xp = np.empty_like(x)
    lib().or_departure(x.shape[1], x.shape[0], _p(x, _f64), _p(u, _f64), float(dt),
                       _p(xp, _f64))
    return xp


def locate_bruteforce(v0, M, pts, eps=EPS):
    v0, M, pts = _f(v0), _f(M), _f(pts)
    host = np.empty(pts.shape[0], dtype=np.int32)
    lib().or_locate_bruteforce(v0.shape[1], v0.shape[0], _p(v0, _f64), _p(M, _f64),
                               pts.shape[0], _p(pts, _f64), eps, _p(host, _i32))
    return host


def locate_bucketed(xyz, conn, v0, M, pts, eps=EPS, g=None):
    xyz, conn, v0, M, pts = _f(xyz), _i(conn), _f(v0), _f(M), _f(pts)
    dim = xyz.shape[1]
    if g is None:
        per_cell = 4.0 if dim == 2 else 24.0
        g = max(1, int(round((conn.shape[0] / per_cell) ** (1.0 / dim))))
    host = np.empty(pts.shape[0], dtype=np.int32)
    rc = lib().or_locate_bucketed(dim, xyz.shape[0], _p(xyz, _f64), conn.shape[0],
                                  _p(conn, _i32), _p(v0, _f64), _p(M, _f64), pts.shape[0],
                                  _p(pts, _f64), eps, int(g), _p(host, _i32))
    if rc:
        raise MemoryError("oracle bucket grid")
    return host


def walk(v0, M, nbr, pts, start, eps=EPS, cap=None):
    v0, M, nbr, pts, start = _f(v0), _f(M), _i(nbr), _f(pts), _i(start)
    dim = v0.shape[1]
    n = pts.shape[0]
    if cap is None:
        cap = step_cap(dim, v0.shape[0])
    end = np.empty(n, dtype=np.int32)
    it = np.empty(n, dtype=np.int32)
    reason = np.empty(n, dtype=np.uint8)
    lib().or_walk(dim, _p(v0, _f64), _p(M, _f64), _p(nbr, _i32), n, _p(pts, _f64),
                  _p(start, _i32), eps, int(cap), _p(end, _i32), _p(it, _i32),
                  _p(reason, _u8))
    return end, it, reason


def node_elements(n_v, conn):
    conn = _i(conn)
    dim = conn.shape[1] - 1
    out = np.empty(n_v, dtype=np.int32)
    lib().or_node_elements(dim, n_v, conn.shape[0], _p(conn, _i32), _p(out, _i32))
    return out


def step_cap(dim, n_e):
    """Step cap 8 * n_e^(1/d) + 64 (the paper sets none; Algorithm 1 may cycle
    on non-Delaunay meshes)."""
    return int(8 * round(n_e ** (1.0 / dim)) + 64)


# ---------------------------------------------------------------------------
# ASG grid (Sec. 1, 2.3)
# ---------------------------------------------------------------------------

def bbox(xyz):
    xyz = _f(xyz)
    return xyz.min(axis=0).copy(), xyz.max(axis=0).copy()


def grid_centres(lo, hi, g):
    lo, hi, g = _f(lo), _f(hi), _i(g)
    dim = lo.shape[0]
    n = int(np.prod(g.astype(np.int64)))
    out = np.empty((n, dim))
    lib().or_grid_centres(dim, _p(lo, _f64), _p(hi, _f64), _p(g, _i32), _p(out, _f64))
    return out


def grid_cells(lo, hi, g, pts):
    lo, hi, g, pts = _f(lo), _f(hi), _i(g), _f(pts)
    dim = lo.shape[0]
    out = np.empty(pts.shape[0], dtype=np.int64)
    lib().or_grid_cells(dim, _p(lo, _f64), _p(hi, _f64), _p(g, _i32), pts.shape[0],
                        _p(pts, _f64), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)))
    return out


def p1_interpolate(conn, v0, M, u_nodal, pts, host):
    conn, v0, M, u_nodal, pts, host = _i(conn), _f(v0), _f(M), _f(u_nodal), _f(pts), _i(host)
    dim = v0.shape[1]
    out = np.empty((pts.shape[0], dim))
    lib().or_p1_interpolate(dim, _p(conn, _i32), _p(v0, _f64), _p(M, _f64),
                            _p(u_nodal, _f64), pts.shape[0], _p(pts, _f64),
                            _p(host, _i32), _p(out, _f64))
    return out


# ---------------------------------------------------------------------------
# whole mesh + track
# ---------------------------------------------------------------------------

class Mesh:
    """The oracle's own view of a mesh: neighbours, inverse-affine form,
    plain-SNS starts and the ASG seed grid (host of every cell centre)."""

    def __init__(self, xyz, conn, grid=None, brute_limit=20000, pred_stride=1):
        self.xyz = _f(xyz)
        self.conn = _i(conn)
        self.dim = self.xyz.shape[1]
        self.n_v = self.xyz.shape[0]
        self.n_e = self.conn.shape[0]
        self.nbr = neighbors(self.dim, self.conn)
        self.v0, self.M = inverse_affine(self.xyz, self.conn)
        self.node_elem = node_elements(self.n_v, self.conn)
        self.cap = step_cap(self.dim, self.n_e)
        self.brute = self.n_e <= brute_limit
        self.lo, self.hi = bbox(self.xyz)
        if grid is None:
            grid = default_grid(self.n_v, self.dim)
        self.grid = _i(np.broadcast_to(np.asarray(grid), (self.dim,)))
        self._seed = None
        self.set_pred_stride(pred_stride)

    def set_pred_stride(self, p):
        """The predictor grid (Sec. 2.3: the ASG pools several elements into
        each Cartesian cell): cells of p^d ASG cells, p odd, aligned at lo;
        grid // p cells per axis of size ((hi - lo) / grid) * p. A point past
        the last whole cell belongs to the last one."""
        if p < 1 or p % 2 == 0:
            raise ValueError("predictor stride must be odd and >= 1")
        self.pred_stride = int(p)
        self.pgrid = np.maximum(self.grid // p, 1).astype(np.int32)
        self.ps = ((self.hi - self.lo) / self.grid) * float(p)

    def pred_centres(self):
        """Centres lo + (i + 0.5) * ps of the predictor cells, x fastest."""
        axes = [(np.arange(g) + 0.5) * s for g, s in zip(self.pgrid, self.ps)]
        mesh = np.meshgrid(*axes[::-1], indexing="ij")[::-1]
        return np.stack([self.lo[k] + mesh[k].ravel() for k in range(self.dim)], axis=1)

    def pred_cells(self, pts):
        """Predictor cell of each point: floor((x - lo) / ps) per axis, clamped
        to [0, pgrid - 1] (NaN -> 0), flattened x fastest."""
        pts = _f(pts)
        t = np.floor((pts - self.lo) / self.ps)
        t = np.where(t >= 0.0, t, 0.0)
        t = np.minimum(t, (self.pgrid - 1).astype(np.float64)).astype(np.int64)
        c = np.zeros(pts.shape[0], dtype=np.int64)
        for k in range(self.dim - 1, -1, -1):
            c = c * int(self.pgrid[k]) + t[:, k]
        return c

    def cnn_origin_cells(self, x, dhat):
        """Algorithm 2's origin under reading R23 (single precision; the paper
        fixes none and the origin only chooses the start element): x
        truncated toward zero to float32, its predictor cell, y = x + dhat *
        ps with dhat the prediction at that cell, and the ASG cell of y. All
        arithmetic in float32, each operation rounded to nearest; the grid
        origin, cell sizes and their inverses are the float64 values rounded
        to float32. Returns (predictor cells, ASG cells of y)."""
        xt = trunc_f32(x)
        lo = self.lo.astype(np.float32)
        pinv = (1.0 / self.ps).astype(np.float32)
        pc = np.zeros(xt.shape[0], dtype=np.int64)
        for k in range(self.dim - 1, -1, -1):
            pc = pc * int(self.pgrid[k]) + cell_f32(xt[:, k], lo[k], pinv[k], int(self.pgrid[k]))
        d = np.asarray(dhat, dtype=np.float32).reshape(-1, self.dim)[pc]
        ps = self.ps.astype(np.float32)
        inv = (1.0 / ((self.hi - self.lo) / self.grid)).astype(np.float32)
        c = np.zeros(xt.shape[0], dtype=np.int64)
        for k in range(self.dim - 1, -1, -1):
            y = xt[:, k] + d[:, k] * ps[k]
            c = c * int(self.grid[k]) + cell_f32(y, lo[k], inv[k], int(self.grid[k]))
        return pc, c

    def locate(self, pts, eps=EPS):
        if self.brute:
            return locate_bruteforce(self.v0, self.M, pts, eps)
        return locate_bucketed(self.xyz, self.conn, self.v0, self.M, pts, eps)

    @property
    def seed(self):
        """seed[c] = host of the centre of ASG cell c (or -1)."""
        if self._seed is None:
            self._seed = self.locate(grid_centres(self.lo, self.hi, self.grid))
        return self._seed

    def cells(self, pts):
        return grid_cells(self.lo, self.hi, self.grid, pts)

    def centroids(self):
        return self.xyz[self.conn].mean(axis=1)

    def track(self, x, u, dt, start=None, mode="sns", dhat=None):
        """Full path for every particle: departure point, start element,
        Algorithm 1 walk, exact host and status.

        mode 'sns': start = the given start (user ids) or the node's element;
        'asg': start = seed grid cell of x_p itself; 'cnn': start = seed grid
        cell of x + dhat * ps (dhat the prediction at every predictor cell, in
        predictor cell units, ps the predictor cell size; single precision,
        see cnn_origin_cells). A seed of -1 falls back to the plain start.
        Returns dict of host, path_len, status, start, xp."""
        x, u = _f(x), _f(u)
        n = x.shape[0]
        xp = departure(x, u, dt)
        if start is None:
            if n != self.n_v:
                raise ValueError("start needed unless the particles are the mesh nodes")
            plain = self.node_elem.copy()
        else:
            plain = _i(start).copy()
        if mode == "sns":
            st = plain
        elif mode == "asg":
            c = self.cells(xp)
            s = self.seed[c]
            st = np.where(s >= 0, s, plain).astype(np.int32)
        elif mode == "cnn":
            # dhat: the prediction at every predictor cell, in cell units
            _, c = self.cnn_origin_cells(x, dhat)
            s = self.seed[c]
            st = np.where(s >= 0, s, plain).astype(np.int32)
        else:
            raise ValueError(mode)
        end, it, reason = walk(self.v0, self.M, self.nbr, xp, st, cap=self.cap)
        host = self.locate(xp)
        status = np.where(reason == CONTAINED, ST_FOUND,
                          np.where(host < 0, ST_OUTSIDE, ST_FALLBACK)).astype(np.uint8)
        finite = np.isfinite(xp).all(axis=1)
        nostart = finite & (st < 0)
        it = np.where(nostart, 0, it).astype(np.int32)
        status[~finite] = ST_INVALID
        host = np.where(finite, host, -1).astype(np.int32)
        it[~finite] = 0
        return dict(host=host, path_len=it, status=status, start=st, xp=xp,
                    end=end, reason=reason)


def trunc_f32(x):
    """x truncated toward zero to float32: the significand cut to 24 bits;
    magnitudes below 2^-126 give a signed zero, finite magnitudes of 2^128 and
    more a signed infinity; infinities and NaN stay what they are."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = x.view(np.uint64)
    e = ((b >> np.uint64(52)) & np.uint64(0x7ff)).astype(np.int64) - 1023
    t = (b & ~np.uint64((1 << 29) - 1)).view(np.float64)
    neg = np.signbit(x)
    with np.errstate(over="ignore"):
        out = t.astype(np.float32)
    out = np.where(e < -126, np.where(neg, np.float32(-0.0), np.float32(0.0)), out)
    big = (e > 127) & np.isfinite(x)
    out = np.where(big, np.where(neg, np.float32(-np.inf), np.float32(np.inf)), out)
    return out.astype(np.float32)


def cell_f32(v, lo, inv, g):
    """floor((v - lo) * inv) in float32 (each operation rounded to nearest),
    clamped to [0, g - 1]; negative and NaN quotients give 0."""
    v = np.asarray(v, dtype=np.float32)
    q = (v - np.float32(lo)) * np.float32(inv)
    with np.errstate(invalid="ignore"):
        f = np.floor(q)
        ok = q >= np.float32(0.0)
    return np.where(ok, np.minimum(f, np.float32(g - 1)), np.float32(0.0)).astype(np.int64)


def default_grid(n_v, dim):
    """Default ASG resolution per axis: round(n_v^(1/d)) - 1, at least 1."""
    return max(1, int(round(n_v ** (1.0 / dim))) - 1)
