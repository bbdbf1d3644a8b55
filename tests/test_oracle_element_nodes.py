"""Pins of the per-(element, node) particle layout (Sec. 2.1, Eq. 4: each
element's nodes are traced back from that element) in the oracle.

- The layout itself: n = (d + 1) n_e particles, element-major, each at its
  node with the node's velocity, starting from its own element.
- dt = 0: the particle sits on a vertex of its start element, so the walk
  stops there at once (I_t = 1) and the exact host is the lowest-id element
  owning the vertex: the plain-SNS node start K_m of Eq. 4.
- dt > 0: a pair's departure point equals its node's, so its host (unique,
  whatever the start) equals the host of the node particle.
"""

import numpy as np
import pytest

import oracle
from workloads import make_case, element_node_particles


@pytest.fixture(scope="module", params=[("tg2d", 31), ("abc3d", 7)])
def setup(request):
    name, n_side = request.param
    c = make_case(name, n_side=n_side, cfl=6)
    return c, oracle.Mesh(c.xyz, c.conn)


def test_layout(setup):
    c, _ = setup
    x, u, start = element_node_particles(c)
    assert x.shape == ((c.dim + 1) * c.n_elements, c.dim) and u.shape == x.shape
    e = np.arange(c.n_elements)
    assert np.array_equal(start.reshape(c.n_elements, c.dim + 1), np.repeat(e[:, None], c.dim + 1, 1))
    for i in range(c.dim + 1):
        assert np.array_equal(x[i::c.dim + 1], c.xyz[c.conn[:, i]])
        assert np.array_equal(u[i::c.dim + 1], c.u[c.conn[:, i]])


def test_zero_step_ends_at_the_node_start(setup):
    c, om = setup
    x, u, start = element_node_particles(c)
    r = om.track(x, u, 0.0, start=start, mode="sns")
    assert (r["path_len"] == 1).all() and (r["status"] == 0).all()
    assert np.array_equal(r["host"], om.node_elem[c.conn.reshape(-1)])


def test_pair_hosts_are_node_hosts(setup):
    c, om = setup
    x, u, start = element_node_particles(c)
    pair = om.track(x, u, c.dt, start=start, mode="sns")
    node = om.track(c.x, c.u, c.dt, mode="sns")
    assert np.array_equal(pair["host"], node["host"][c.conn.reshape(-1)])
    assert np.array_equal(pair["status"] == 1, node["status"][c.conn.reshape(-1)] == 1)
