"""Multi-process path on the CPU (gloo, world size 2).

Each rank locates its slice of the particles (here with the oracle, since the
CPU has no GPU) and the job's reductions are the ones bench.py uses: the
union of the slices must give the single-process result, the time is the
slowest rank's and the particle count the sum.
"""

import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2412_18379_gb300.shard import shard_range


@pytest.mark.parametrize("n,world", [(0, 1), (1, 2), (10, 3), (1002001, 8), (7, 7), (5, 8)])
def test_shard_range_partitions(n, world):
    ranges = [shard_range(n, r, world) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == n
    for (a, b), (c, d) in zip(ranges, ranges[1:]):
        assert b == c
    sizes = [b - a for a, b in ranges]
    assert max(sizes) - min(sizes) <= 1 and sum(sizes) == n


def test_shard_range_rejects_bad_arguments():
    for args in [(10, 2, 2), (10, -1, 2), (10, 0, 0), (-1, 0, 1)]:
        with pytest.raises(ValueError):
            shard_range(*args)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    import oracle
    from paper_2412_18379_gb300.shard import max_over_ranks, sum_over_ranks
    from workloads import make_case
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        c = make_case("tg2d", n_side=41, cfl=4.0)
        mesh = oracle.Mesh(c.xyz, c.conn)
        start = mesh.node_elem
        lo, hi = shard_range(c.n_particles, rank, world)
        r = mesh.track(c.x[lo:hi], c.u[lo:hi], c.dt, start[lo:hi], mode="sns")
        parts = [None] * world
        dist.all_gather_object(parts, (lo, hi, r["host"], r["path_len"], r["status"]))
        slowest = max_over_ranks(1.0 + rank)
        total = sum_over_ranks(hi - lo)
        if rank == 0:
            np.savez(os.path.join(out_dir, "gathered.npz"),
                     lo=np.array([p[0] for p in parts]), hi=np.array([p[1] for p in parts]),
                     host=np.concatenate([p[2] for p in parts]),
                     path_len=np.concatenate([p[3] for p in parts]),
                     status=np.concatenate([p[4] for p in parts]),
                     slowest=slowest, total=total)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo_union_equals_single_process(tmp_path):
    import oracle
    from workloads import make_case
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    g = np.load(tmp_path / "gathered.npz")
    c = make_case("tg2d", n_side=41, cfl=4.0)
    mesh = oracle.Mesh(c.xyz, c.conn)
    full = mesh.track(c.x, c.u, c.dt, mesh.node_elem, mode="sns")
    assert list(g["lo"]) == [0, g["hi"][0]] and g["hi"][1] == c.n_particles
    for k in ("host", "path_len", "status"):
        assert np.array_equal(g[k], full[k]), k
    assert float(g["slowest"]) == 2.0 and int(g["total"]) == c.n_particles
