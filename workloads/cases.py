"""Named workloads: mesh + one particle per mesh node + velocity + time step.

  rotation2d  51 x 51 jittered (+-0.3h, seed 1) Delaunay square, solid-body
              rotation about (0.5, 0.5), CFL 2; ~5k triangles, 2,601 particles.
  tg2d        n x n jittered (+-0.3h, seed 2) Delaunay square, Taylor-Green,
              CFL swept; n = 1001 gives ~2.0M triangles and ~1.0M particles.
  abc3d       n^3 jittered (+-0.1h, seed 3) Kuhn cube, ABC flow (A=B=C=1),
              CFL swept; n = 101 gives 6.0M tetrahedra and 1,030,301 particles.
  modes2d /   random 8-mode Fourier fields (training and serving inputs).
  modes3d

Each particle sits at a mesh node x with the nodal velocity u = u(x); its
departure point is x - u*dt, formed by the code under test.
"""

from dataclasses import dataclass

import numpy as np

from .meshes import mesh_2d, mesh_2d_hole, mesh_3d, mesh_3d_sphere
from .fields import (rotation, taylor_green, abc_flow, fourier_modes_2d,
                     fourier_modes_3d, dt_for_cfl)


@dataclass
class Case:
    name: str
    dim: int
    xyz: np.ndarray      # [n_v, dim] float64 vertex coordinates
    conn: np.ndarray     # [n_e, dim+1] int32 connectivity (user element ids = row index)
    h: float             # lattice spacing
    x: np.ndarray        # [n, dim] float64 particle positions (the mesh nodes)
    u: np.ndarray        # [n, dim] float64 velocity at the particles
    dt: float
    cfl: float

    @property
    def n_particles(self):
        return self.x.shape[0]

    @property
    def n_elements(self):
        return self.conn.shape[0]


def make_case(name, cfl=None, n_side=None, seed=None, field_seed=None):
    if name == "rotation2d":
        n_side = n_side or 51
        xyz, conn, h = mesh_2d(n_side, 0.3, 1 if seed is None else seed)
        u = rotation(xyz)
        cfl = 2.0 if cfl is None else cfl
    elif name == "tg2d":
        n_side = n_side or 1001
        xyz, conn, h = mesh_2d(n_side, 0.3, 2 if seed is None else seed)
        u = taylor_green(xyz)
        cfl = 8.0 if cfl is None else cfl
    elif name == "abc3d":
        n_side = n_side or 101
        xyz, conn, h = mesh_3d(n_side, 0.1, 3 if seed is None else seed)
        u = abc_flow(xyz)
        cfl = 8.0 if cfl is None else cfl
    elif name == "modes2d":
        n_side = n_side or 201
        xyz, conn, h = mesh_2d(n_side, 0.3, 100 if seed is None else seed)
        u = fourier_modes_2d(xyz, 1000 if field_seed is None else field_seed)
        cfl = 8.0 if cfl is None else cfl
    elif name == "hole2d":
        # uniform flow past a disc-shaped hole: the walks of the nodes behind
        # the hole meet its boundary, and some departure points fall in it
        n_side = n_side or 101
        xyz, conn, h = mesh_2d_hole(n_side, 0.1, 0.3, 7 if seed is None else seed)
        u = np.ascontiguousarray(np.broadcast_to(np.array([0.94, 0.34]), xyz.shape))
        cfl = 16.0 if cfl is None else cfl
    elif name == "sphere3d":
        # uniform flow past a ball-shaped hole in the cube (the geometry of
        # the paper's second benchmark): walks behind the ball meet its
        # boundary, and some departure points fall into it
        n_side = n_side or 51
        xyz, conn, h = mesh_3d_sphere(n_side, 0.2, 0.1, 11 if seed is None else seed)
        d = np.array([0.90, 0.35, 0.25])
        u = np.ascontiguousarray(np.broadcast_to(d / np.linalg.norm(d), xyz.shape))
        cfl = 0.16 / h if cfl is None else cfl      # a displacement of 0.16

    elif name == "modes3d":
        n_side = n_side or 41
        xyz, conn, h = mesh_3d(n_side, 0.1, 200 if seed is None else seed)
        u = fourier_modes_3d(xyz, 2000 if field_seed is None else field_seed)
        cfl = 8.0 if cfl is None else cfl
    else:
        raise ValueError("unknown workload %r" % name)
    dim = xyz.shape[1]
    dt = dt_for_cfl(u, h, cfl)
    x = np.array(xyz, dtype=np.float64, copy=True)
    return Case(name=name, dim=dim, xyz=xyz, conn=conn, h=h, x=x,
                u=np.ascontiguousarray(u), dt=dt, cfl=cfl)


def element_node_particles(case):
    """One particle per (element, local node) pair, the characteristic-tracing
    layout of an L-G step (Sec. 2.1, Eq. 4: every element's nodes are traced
    back from that element): n = (d + 1) * n_elements particles, ordered
    element-major. Returns (x, u, start): the node's position and velocity,
    and the owning element's user id as the plain-SNS start."""
    nodes = case.conn.reshape(-1)
    x = np.ascontiguousarray(case.xyz[nodes])
    u = np.ascontiguousarray(case.u[nodes])
    start = np.repeat(np.arange(case.n_elements, dtype=np.int32), case.dim + 1)
    return x, u, start
