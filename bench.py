#!/usr/bin/env python3
"""Particle-location benchmark: particles located per second and walk lengths.

Workload (default): the 1001 x 1001 jittered Delaunay unit square (~2.0M
triangles), one particle per node (1,002,001), Taylor-Green velocity at
CFL 8. A step locates every particle once through the library's C ABI
(departure point, start element, Algorithm 1 walk, exact canonicalisation);
inputs are resident in HBM, and L2 is flushed (a 256 MB write) before every
timed step. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--cfl C] [--mode M]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores
"""

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "tg2d": dict(name="tg2d", n_side=1001,
                 desc="2-D unit square, 1001x1001 lattice jittered +-0.3h (seed 2), "
                      "Delaunay (~2.0M triangles), Taylor-Green u, one particle per node"),
    "abc3d": dict(name="abc3d", n_side=101,
                  desc="3-D unit cube, 101^3 lattice jittered +-0.1h (seed 3), 6 Kuhn "
                       "tets per cell (6.0M tets), ABC flow, one particle per node"),
}

REC_ALG_BYTES = {2: 60, 3: 112}      # v0 + M + neighbours per walk step


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2412_18379_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


WALK_SOURCES = ("walk.cu", "walk_common.cuh", "internal.h")


def ncu_traffic(dim):
    """DRAM bytes per launch of the walk kernel from the committed ncu summary,
    if it was taken on the current source; else None."""
    prof = os.path.join(ROOT, "profiles", "walk_kernel_tg2d_ncu.md" if dim == 2
                        else "walk_kernel_abc3d_ncu.md")
    if not os.path.exists(prof):
        return None
    sha = source_sha(WALK_SOURCES)
    vals = {}
    for line in open(prof):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != sha:
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join("/tmp", "bench_clocks_%d_%d.csv" % (os.getpid(), index))

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "25"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx = max(mx, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_oracle_rate(case, mode, sample_n, seed=0):
    """The oracle as it stands (single-threaded C through ctypes) on a bounded
    sample of the workload's particles; returns particles/s and the sample."""
    import oracle
    om = oracle.Mesh(case.xyz, case.conn)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(case.n_particles, size=min(sample_n, case.n_particles),
                             replace=False))
    start = om.node_elem[idx]
    t0 = time.perf_counter()
    r = om.track(case.x[idx], case.u[idx], case.dt, start=start,
                 mode="sns" if mode == "cnn" else mode)
    dt = time.perf_counter() - t0
    return idx.size / dt, dt, r


def run_reference(args):
    r, w, _ = rank_info()
    if r != 0:
        return 0
    from workloads import make_case
    wl = WORKLOADS[args.workload]
    case = make_case(wl["name"], cfl=args.cfl, n_side=wl["n_side"])
    sample = args.ref_sample
    times = []
    for i in range(args.warmup + args.steps):
        rate, dt, _ = cpu_oracle_rate(case, args.mode, sample, seed=i)
        if i >= args.warmup:
            times.append(dt)
    per_step = float(np.mean(times))
    value = sample / per_step
    line = {
        "impl": "reference", "metric": "particles located/s", "value": value,
        "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"] + ", CFL %g" % args.cfl, "mode": "sns",
                   "sample_particles": sample},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": 1, "kind": "oracle",
                         "sample": "%d particles drawn from the workload per step" % sample},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg2d", choices=sorted(WORKLOADS))
    ap.add_argument("--cfl", type=float, default=8.0)
    ap.add_argument("--mode", default="sns", choices=["sns", "asg"])
    ap.add_argument("--ref-sample", type=int, default=200000)
    ap.add_argument("--cpu-sample", type=int, default=200000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="time the main mode only (no other modes, e2e or CPU leg); "
                         "used for profiler captures")
    args = ap.parse_args()
    if args.quick:
        args.no_cpu_baseline = True
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    rank, world, lrank = rank_info()
    torch.cuda.set_device(lrank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2412_18379_gb300 as cs
    from paper_2412_18379_gb300 import build
    from workloads import make_case

    if rank == 0 or world == 1:
        build.build()
    if dist is not None:
        dist.barrier()
    wl = WORKLOADS[args.workload]
    case = make_case(wl["name"], cfl=args.cfl, n_side=wl["n_side"])
    dim = case.dim
    ctx = cs.Context(lrank)
    mesh = ctx.upload_mesh(case.xyz, case.conn)
    info = mesh.info()
    dev = torch.device("cuda", lrank)
    x = torch.from_numpy(case.x).to(dev)
    u = torch.from_numpy(case.u).to(dev)
    n = case.n_particles
    out = dict(host=torch.empty(n, dtype=torch.int32, device=dev),
               path_len=torch.empty(n, dtype=torch.int32, device=dev),
               status=torch.empty(n, dtype=torch.uint8, device=dev))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(mode):
        ctx.track(mesh, x, u, case.dt, mode=mode, out=out, stream=stream)

    def timed(mode, steps, warmup):
        for _ in range(warmup):
            step(mode)
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        ctx.profile(True)
        ctx.profile_read(reset=True)
        l0 = ctx.launches
        total = 0.0
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for i in range(steps):
            flush.fill_(i & 0xff)
            ev[i][0].record(stream)
            step(mode)
            ev[i][1].record(stream)
        torch.cuda.synchronize()
        for a, b in ev:
            total += a.elapsed_time(b)
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        launches = ctx.launches - l0
        if dist is not None:
            t = torch.tensor([total], device=dev, dtype=torch.float64)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            total = float(t.item())
            dist.barrier()
        torch.cuda.synchronize()
        st = ctx.stats(out["path_len"], out["status"])
        return total, prof, launches, st

    sampler = ClockSampler(lrank)
    sampler.start()
    total_ms, prof, launches, st = timed(args.mode, args.steps, args.warmup)
    clocks = sampler.stop()
    ms_per_step = total_ms / args.steps
    value = world * n / (ms_per_step * 1e-3)
    mean_it = st["sum"] / n

    # the other start rules, for the same workload
    others = {}
    for mode in (("sns", "asg") if not args.quick else (args.mode,)):
        if mode == args.mode:
            others[mode] = dict(particles_per_s=value / world, ms_per_step=ms_per_step,
                                mean_path_len=mean_it, max_path_len=st["max"])
            continue
        t2, _, _, st2 = timed(mode, max(3, args.steps // 2), 3)
        mps = t2 / max(3, args.steps // 2)
        others[mode] = dict(particles_per_s=n / (mps * 1e-3), ms_per_step=mps,
                            mean_path_len=st2["sum"] / n, max_path_len=st2["max"])

    # roofline of the walk kernel: algorithmic bytes / event-timed duration
    walk_launches, walk_ms = prof["walk"]
    alg_bytes = n * (16 * dim + 13) + st["sum"] * REC_ALG_BYTES[dim]
    achieved = alg_bytes / (walk_ms / walk_launches * 1e-3) / 1e9 if walk_launches else 0.0
    peak, peak_kind = peaks()
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": ncu_traffic(dim),
                "peak_source": peak_kind + " (MEASURED_PEAKS.json hbm_gbs)"
                if peak_kind == "measured" else "fallback 6.8 TB/s",
                "kernel": "walk_kernel<%d>" % dim,
                "kernel_ms": walk_ms / max(1, walk_launches),
                "algorithmic_bytes_per_launch": alg_bytes}

    # end to end through the host-pointer entry point (pinned buffers)
    xh = torch.from_numpy(case.x).pin_memory()
    uh = torch.from_numpy(case.u).pin_memory()
    hout = dict(host=torch.empty(n, dtype=torch.int32).pin_memory(),
                path_len=torch.empty(n, dtype=torch.int32).pin_memory(),
                status=torch.empty(n, dtype=torch.uint8).pin_memory())
    for _ in range(0 if args.quick else 3):
        ctx.track_host(mesh, xh, uh, case.dt, mode=args.mode, out=hout)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e2e_steps = max(3, args.steps // 2) if not args.quick else 1
    for _ in range(e2e_steps):
        ctx.track_host(mesh, xh, uh, case.dt, mode=args.mode, out=hout)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if dist is not None:
        t = torch.tensor([e2e_s], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e = {"value": world * n / e2e_s, "unit": "particles/s",
           "h2d_bytes_per_step": n * dim * 16, "d2h_bytes_per_step": n * 9,
           "entry_point": "cs_track_host"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, dt_cpu, _ = cpu_oracle_rate(case, args.mode, args.cpu_sample)
        cpu = {"value": rate, "unit": "particles/s", "cores": 1, "kind": "oracle",
               "sample": "%d of the %d particles (seeded draw), oracle.Mesh.track: "
                         "departure + Algorithm 1 walk + exact bucketed host, %.1f s"
                         % (args.cpu_sample, n, dt_cpu)}

    if rank == 0:
        line = {
            "metric": "particles located/s", "value": value, "unit": "particles/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl["desc"] + ", CFL %g" % args.cfl, "mode": args.mode,
                       "n_particles": n, "n_elements": case.n_elements,
                       "asg_grid": info["asg_grid"], "l2": "flushed by a 256 MB write "
                       "before every timed step", "parallelism": "replicas" if world > 1
                       else "1 GPU"},
            "mean_path_len": mean_it, "max_path_len": st["max"],
            "status_counts": [st["found"], st["outside"], st["fallback"], st["invalid"]],
            "modes": others,
            "stage_ms_per_step": {k: v[1] / max(1, v[0]) for k, v in prof.items() if v[0]},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": launches, "clocks": clocks,
        }
        print(json.dumps(line))
    mesh.release()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
