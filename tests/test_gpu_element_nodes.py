"""Per-(element, node) particles and multi-step time loops on the GPU.

The characteristic tracing of an L-G step follows every element's nodes back
from that element (Sec. 2.1, Eq. 4), so the particle set is one particle per
(element, local node) pair, n = (d + 1) n_e, each starting from its own
element. Over a time loop, a step's hosts are the natural starts of the next
step. Both go through the C ABI with explicit starts and must match the
oracle bit for bit: hosts, path lengths, statuses and start elements.
"""

import numpy as np
import pytest

import oracle
from workloads import make_case, element_node_particles

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import paper_2412_18379_gb300 as cs
    from paper_2412_18379_gb300 import build
    build.build()
    c = cs.Context(0)
    yield c
    c.close()


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _run(ctx, mesh, x, u, dt, start, mode="sns"):
    import torch
    out = ctx.track(mesh, _dev(x), _dev(u), dt, start=_dev(start.astype(np.int32)), mode=mode,
                    start_out=True)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check(got, want, what):
    st = np.where(want["path_len"] > 0, want["start"], -1)
    for k, ref in (("host", want["host"]), ("path_len", want["path_len"]),
                   ("status", want["status"]), ("start", st)):
        bad = np.nonzero(got[k] != ref)[0]
        assert bad.size == 0, "%s %s differs at %d particles, first %s" % (what, k, bad.size, bad[:5])


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 101, "cfl": 8}),
                                     ("abc3d", {"n_side": 11, "cfl": 8}),
                                     ("hole2d", {"n_side": 61}),
                                     ("sphere3d", {"n_side": 21})])
def test_element_node_particles(ctx, name, kw):
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    x, u, start = element_node_particles(c)
    for mode in ("sns", "asg"):
        got = _run(ctx, mesh, x, u, c.dt, start, mode)
        _check(got, om.track(x, u, c.dt, start=start, mode=mode), "%s %s" % (name, mode))
    mesh.release()


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 101, "cfl": 4}),
                                     ("abc3d", {"n_side": 11, "cfl": 4})])
def test_time_loop_with_previous_hosts_as_starts(ctx, name, kw):
    """Four steps of an L-G loop: the particles stay at their nodes, the
    velocity field changes slowly (here it grows by 10% a step, u_t =
    (1 + t/10) u_0, the same FP64 products on both sides), and a step's
    hosts start the next step's walks. Every step matches the oracle's loop;
    from the second step on the walks are much shorter than from the
    element, since the previous host lies next to the new departure point."""
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    om = oracle.Mesh(c.xyz, c.conn, grid=mesh.info()["asg_grid"])
    x, u0, start = element_node_particles(c)
    first = None
    for t in range(4):
        u = u0 * (1.0 + 0.1 * t)
        got = _run(ctx, mesh, x, u, c.dt, start)
        want = om.track(x, u, c.dt, start=start, mode="sns")
        _check(got, want, "%s step %d" % (name, t))
        mean = got["path_len"][got["path_len"] > 0].mean()
        if t == 0:
            first = mean
        else:
            assert mean < 0.5 * first, (t, mean, first)
        start = got["host"]
    mesh.release()
