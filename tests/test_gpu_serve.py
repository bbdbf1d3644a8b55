"""Serving: continuous batching over resident meshes, fields and predictor.

Each request's result must be the same alone and in the mix (bit for bit:
the walk is exact and the predictor deterministic), requests must overlap on
the GPU, admission must respect the arena, and an oversized request must be
refused with an error instead of blocking the queue.
"""

import numpy as np
import pytest

from workloads import make_case
from workloads.weights import init_weights
from workloads.fields import dt_for_cfl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    import paper_2412_18379_gb300 as cs
    from paper_2412_18379_gb300 import build
    build.build()
    ctx = cs.Context(0)
    ctx.load_predictor(2, init_weights(2, 5))
    ctx.load_predictor(3, init_weights(3, 5))
    meshes = []
    for name, kw in [("tg2d", {"n_side": 201}), ("modes2d", {"n_side": 301}),
                     ("abc3d", {"n_side": 21})]:
        c = make_case(name, **kw)
        m = ctx.upload_mesh(c.xyz, c.conn)
        m.set_predictor_grid(3)
        f = ctx.upload_field(m, c.u)                       # resident field
        meshes.append((c, m, m.node_start_elements(), f))
    # uploaded before serving starts (meshes are fixed while serving)
    big = make_case("tg2d", n_side=401)
    mb = ctx.upload_mesh(big.xyz, big.conn)
    torch.cuda.synchronize()
    yield ctx, meshes, (big, mb)
    ctx.close()


def _requests(meshes, count, seed):
    import torch
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        c, m, node_elem, f = meshes[rng.integers(len(meshes))]
        n = int(np.exp(rng.uniform(np.log(500), np.log(c.n_particles))))
        idx = np.sort(rng.choice(c.n_particles, size=n, replace=False))
        x = torch.from_numpy(np.ascontiguousarray(c.x[idx])).pin_memory()
        u = torch.from_numpy(np.ascontiguousarray(c.u[idx])).pin_memory()
        st = torch.from_numpy(np.ascontiguousarray(node_elem[idx])).pin_memory()
        dt = dt_for_cfl(c.u, c.h, rng.uniform(1.0, 16.0))
        mode = ["sns", "asg", "cnn"][i % 3]
        reqs.append((m, x, u, st, dt, mode, f))
    return reqs


def _run(ctx, reqs, burst):
    import torch
    outs = [None] * len(reqs)
    if burst:
        # odd requests write into slices of one pinned block the caller owns
        total = sum(int(x.shape[0]) for _, x, *_ in reqs)
        block = dict(host=torch.full((total,), -7, dtype=torch.int32, pin_memory=True),
                     path_len=torch.full((total,), -7, dtype=torch.int32, pin_memory=True),
                     status=torch.full((total,), 77, dtype=torch.uint8, pin_memory=True))
        tickets, o = [], 0
        for i, (m, x, u, st, dt, mode, f) in enumerate(reqs):
            n = int(x.shape[0])
            out = {k: v[o:o + n] for k, v in block.items()} if i % 2 else None
            o += n
            tickets.append(ctx.submit(m, x, u, dt, start=st, mode=mode, field=f, out=out))
        modes = [ctx.wait(t) for t, _ in tickets]
        outs = [{k: v.numpy().copy() for k, v in o.items()} for _, o in tickets]
    else:
        modes = []
        for i, (m, x, u, st, dt, mode, f) in enumerate(reqs):
            t, o = ctx.submit(m, x, u, dt, start=st, mode=mode, field=f)
            modes.append(ctx.wait(t))
            outs[i] = {k: v.numpy().copy() for k, v in o.items()}
    return outs, modes


def test_results_same_alone_and_in_the_mix(setup):
    ctx, meshes, _ = setup
    reqs = _requests(meshes, 36, seed=1)
    ctx.serve_start(slots=6, arena_bytes=1 << 30)
    try:
        alone, modes_a = _run(ctx, reqs, burst=False)
        mixed, modes_b = _run(ctx, reqs, burst=True)
        rep = ctx.serve_report()
        trace = ctx.serve_trace()
    finally:
        ctx.serve_stop()
    assert modes_a == modes_b
    for i, (a, b) in enumerate(zip(alone, mixed)):
        for k in ("host", "path_len", "status"):
            assert np.array_equal(a[k], b[k]), (i, k)
    # CNN-SNS requests ran CNN-SNS on their own field, in 2-D (tensor cores)
    # and in 3-D (tile engine)
    for (m, _, _, _, _, mode, _), used in zip(reqs, modes_b):
        if mode == "cnn":
            assert used == 1
    assert {m.dim for (m, _, _, _, _, mode, _) in reqs if mode == "cnn"} == {2, 3}
    # the mix overlapped on the device and the latencies are reported
    assert rep["completed"] == 72 and rep["rejected"] == 0
    assert rep["max_concurrent"] > 1
    assert 0 < rep["p50_ms"] <= rep["p99_ms"] <= rep["max_ms"]
    # the trace holds every request once, in finishing order, with its own
    # size, mesh and start rule, and the report's latencies are its spans
    assert len(trace) == 72
    assert len({r["ticket"] for r in trace}) == 72
    assert sorted(r["n"] for r in trace) == sorted(2 * [int(q[1].shape[0]) for q in reqs])
    assert sorted(r["mesh_id"] for r in trace) == sorted(2 * [q[0].id for q in reqs])
    assert all(r["result"] == 0 and 0 <= r["slot"] < 6 and 1 <= r["in_flight"] <= 6
               and 0 <= r["submit_ms"] <= r["admit_ms"] <= r["done_ms"] for r in trace)
    assert all(a["done_ms"] <= b["done_ms"] for a, b in zip(trace, trace[1:]))
    assert max(r["in_flight"] for r in trace) == rep["max_concurrent"]
    # the device time of a request's stages fits in its admit-to-done span;
    # only CNN-SNS requests run the predictor, and each keeps its own dt
    # (tickets count from 1 in submission order: both runs submit reqs in order)
    for r in trace:
        q = reqs[(r["ticket"] - 1) % len(reqs)]
        assert r["n"] == int(q[1].shape[0]) and r["dt"] == q[4]
        stages = r["h2d_ms"] + r["predict_ms"] + r["walk_ms"] + r["d2h_ms"]
        assert r["h2d_ms"] > 0 and r["walk_ms"] > 0 and r["d2h_ms"] > 0
        assert stages <= r["done_ms"] - r["admit_ms"] + 0.05
        if r["mode_used"] == 1:
            assert r["predict_ms"] > 0
        else:
            assert r["predict_ms"] == 0
    lat = sorted(r["done_ms"] - r["submit_ms"] for r in trace)
    assert abs(lat[-1] - rep["max_ms"]) < 1e-6 and abs(lat[35] - rep["p50_ms"]) < 1e-6
    # the serving results equal the direct host-pointer entry point
    for i in range(6):
        m, x, u, st, dt, mode, f = reqs[i]
        ref = ctx.track_host(m, x.numpy(), u.numpy(), dt, start=st.numpy(), mode=mode, field=f)
        for k in ("host", "path_len", "status"):
            assert np.array_equal(ref[k], alone[i][k]), (i, mode, k)


def test_admission_by_footprint(setup):
    import paper_2412_18379_gb300 as cs
    ctx, meshes, (big, mb) = setup
    c, m, node_elem, _ = meshes[0]
    # an arena that fits about two of these requests at a time
    n = c.n_particles
    per = n * (2 * 2 * 8 + 4 + 4 + 4 + 1 + 4) + 8 * 256
    ctx.serve_start(slots=8, arena_bytes=int(2.5 * per))
    try:
        reqs = [(m, *(__import__("torch").from_numpy(a).pin_memory()
                      for a in (c.x, c.u, node_elem)), c.dt * (1 + i % 4), "sns", None)
                for i in range(10)]
        outs, _ = _run(ctx, reqs, burst=True)       # queues, never deadlocks
        rep = ctx.serve_report()
        assert rep["completed"] == 10 and rep["max_concurrent"] <= 2
        assert rep["peak_bytes"] <= int(2.5 * per)
        # a request that can never fit is refused at once
        import torch
        with pytest.raises(cs.CsError) as e:
            ctx.submit(mb, torch.from_numpy(big.x).pin_memory(),
                       torch.from_numpy(big.u).pin_memory(), big.dt)
        assert e.value.code == -2
        assert ctx.serve_report()["rejected"] == 1
    finally:
        ctx.serve_stop()
