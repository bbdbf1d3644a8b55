"""cs_track_noalloc: the tracking entry point that allocates no device memory.

It serves callers that cannot let a library allocate during a call (a solver
that owns all device memory through its own pool, or a time-step loop that
cannot afford the synchronisation cudaMalloc/cudaFree may bring). Its scratch
is a fixed 256-byte device array inside the library (the walk's work
cursor; the exact searches run inside the walk and need no list), shared by
every call. These tests
call it through the C ABI and compare it with cs_track, which uses the
context's allocated scratch, on two calls in a row (the second call must not
see the first call's leftovers). This file is named to be collected last.
"""

import numpy as np
import pytest

from workloads import make_case

pytestmark = pytest.mark.gpu

N_LIMIT = (1 << 31) - 1     # first n that cs_track and cs_track_noalloc reject


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


@pytest.mark.parametrize("name,kw", [("tg2d", {"n_side": 301, "cfl": 8}),
                                     ("abc3d", {"n_side": 21, "cfl": 12})])
def test_noalloc_matches_track_twice(ctx, name, kw):
    import torch
    c = make_case(name, **kw)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    x, u = _dev(c.x), _dev(c.u)
    n = c.n_particles
    # two calls in a row with different inputs: the shared scratch keeps the
    # first call's contents, which must not leak into the second
    for dt, mode in ((c.dt, "sns"), (c.dt * 3.0, "asg")):
        want = ctx.track(mesh, x, u, dt, mode=mode, start_out=True)
        out = dict(host=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                   path_len=torch.full((n,), -7, dtype=torch.int32, device="cuda"),
                   status=torch.full((n,), 9, dtype=torch.uint8, device="cuda"),
                   start=torch.full((n,), -7, dtype=torch.int32, device="cuda"))
        got = ctx.track_noalloc(mesh, x, u, dt, mode=mode, out=out)
        torch.cuda.synchronize()
        for k in ("host", "path_len", "status", "start"):
            assert torch.equal(got[k], want[k]), (name, dt, mode, k)
    mesh.release()


def test_noalloc_explicit_starts_and_limit(ctx):
    import torch
    import paper_2412_18379_gb300 as cs
    c = make_case("rotation2d")
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    rng = np.random.default_rng(9)
    start = _dev(rng.integers(-1, c.n_elements, size=c.n_particles).astype(np.int32))
    x, u = _dev(c.x), _dev(c.u)
    for _ in range(2):
        want = ctx.track(mesh, x, u, c.dt, start=start)
        got = ctx.track_noalloc(mesh, x, u, c.dt, start=start)
        torch.cuda.synchronize()
        for k in want:
            assert torch.equal(got[k], want[k]), k
    # outside cs_track's range: a clear error, nothing launched or written
    big = torch.zeros((4, 2), dtype=torch.float64, device="cuda")
    h = torch.full((4,), -7, dtype=torch.int32, device="cuda")
    for n in (N_LIMIT, -1):
        rc = ctx.lib.cs_track_noalloc(ctx.h, mesh.id, cs.CS_NO_FIELD, n, big.data_ptr(),
                                      big.data_ptr(), 0.1, start.data_ptr(), cs.CS_SNS,
                                      h.data_ptr(), h.data_ptr(), h.data_ptr(), None, None)
        assert rc == -1                               # CS_EINVAL
        assert "2^31 - 2" in ctx.lib.cs_last_error(ctx.h).decode()
    # CNN-SNS needs a predicted displacement grid this call would have to
    # allocate: refused with a clear error, with or without a loaded predictor
    from workloads.weights import init_weights
    for loaded in (False, True):
        if loaded:
            ctx.load_predictor(2, init_weights(2, 1))
        for n in (0, 4):
            rc = ctx.lib.cs_track_noalloc(ctx.h, mesh.id, cs.CS_NO_FIELD, n, big.data_ptr(),
                                          big.data_ptr(), 0.1, start.data_ptr(), cs.CS_CNN_SNS,
                                          h.data_ptr(), h.data_ptr(), h.data_ptr(), None, None)
            assert rc == -1                           # CS_EINVAL
            assert "CS_CNN_SNS is not supported" in ctx.lib.cs_last_error(ctx.h).decode()
    torch.cuda.synchronize()
    assert (h.cpu().numpy() == -7).all()
    mesh.release()


def test_noalloc_allocates_no_device_memory(ctx):
    """The defining property: with outputs preallocated, a call leaves the
    device's free memory unchanged (measured around a call after a first one,
    so that lazily loaded kernels are already resident), while cs_track's
    first call on a fresh context allocates its scratch."""
    import torch
    import paper_2412_18379_gb300 as cs
    c = make_case("tg2d", n_side=201, cfl=8)
    fresh = cs.Context(0)
    try:
        mesh = fresh.upload_mesh(c.xyz, c.conn)
        x, u = _dev(c.x), _dev(c.u)
        n = c.n_particles
        out = dict(host=torch.empty(n, dtype=torch.int32, device="cuda"),
                   path_len=torch.empty(n, dtype=torch.int32, device="cuda"),
                   status=torch.empty(n, dtype=torch.uint8, device="cuda"))
        fresh.track_noalloc(mesh, x, u, c.dt, out=out)
        torch.cuda.synchronize()
        before = fresh.memory_usage()[0]
        free0 = torch.cuda.mem_get_info()[0]
        for mode in ("sns", "asg"):
            fresh.track_noalloc(mesh, x, u, c.dt, mode=mode, out=out)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert fresh.memory_usage()[0] == before
        # the allocating entry point, for contrast, takes its scratch on first use
        fresh.track(mesh, x, u, c.dt, out=out)
        torch.cuda.synchronize()
        assert fresh.memory_usage()[0] > before
        mesh.release()
    finally:
        fresh.close()


def test_noalloc_three_million_particles(ctx):
    """More particles than any fixed per-particle scratch of 2^21 entries would
    hold: 3.1M particles (the 301^2 Taylor-Green particles, repeated 34 times
    with explicit starts), same bits as cs_track."""
    import torch
    c = make_case("tg2d", n_side=301, cfl=12)
    mesh = ctx.upload_mesh(c.xyz, c.conn)
    reps = 34
    x = _dev(np.tile(c.x, (reps, 1)))
    u = _dev(np.tile(c.u, (reps, 1)))
    start = _dev(np.tile(mesh.node_start_elements(), reps).astype(np.int32))
    assert x.shape[0] > 3_000_000
    want = ctx.track(mesh, x, u, c.dt, start=start, mode="asg", start_out=True)
    got = ctx.track_noalloc(mesh, x, u, c.dt, start=start, mode="asg", start_out=True)
    torch.cuda.synchronize()
    for k in ("host", "path_len", "status", "start"):
        assert torch.equal(got[k], want[k]), k
    # the repeats are the same particles: every copy has the first one's result
    h = got["host"].cpu().numpy().reshape(reps, -1)
    assert (h == h[0]).all()
    mesh.release()
