#!/usr/bin/env python3
"""Particle-location benchmark: particles located per second, walk lengths,
CNN-SNS against plain SNS.

Workload (default): the 1001 x 1001 jittered Delaunay unit square (2.0M
triangles), one particle per node (1,002,001), Taylor-Green velocity at
CFL 8. A step locates every particle once through the library's C ABI.
Plain SNS walks from the node's element; ASG-direct from the seed of the ASG
cell of x_p (a non-learned control); CNN-SNS (Algorithm 2) resamples the
velocity to the ASG grid, runs the predictor on the tensor cores and walks
from the predicted cell. Inputs are resident in HBM and L2 is flushed (a
256 MB write) before every timed step. Before timing, the predictor is
trained on the GPU on pairs generated by plain SNS on random 8-mode fields
of the same mesh (CFL 2-16).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--cfl C] [--mode M]
  python bench.py --impl reference ...   # the CPU oracle, timed on host cores

Prints one JSON line (rank 0).
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
                      "Delaunay (2.0M triangles), Taylor-Green u, one particle per node"),
    "abc3d": dict(name="abc3d", n_side=101,
                  desc="3-D unit cube, 101^3 lattice jittered +-0.1h (seed 3), 6 Kuhn "
                       "tets per cell (6.0M tets), ABC flow, one particle per node"),
}

REC_ALG_BYTES = {2: 60, 3: 112}      # v0 + M + neighbours per walk step
# The FP64 ceiling of the walk: R1's arithmetic has no FMA, so every
# operation takes one FP64 issue slot; GB300's nominal 1.25 TFLOP/s counts an
# FMA as two flops.
FP64_OPS_PEAK_T = 1.25 / 2


def walk_fp64_ops(n, dim, sum_path):
    """FP64 operations of R1's arithmetic for n particles walking sum_path
    element evaluations in all: per particle the departure point (d products,
    d differences); per evaluation delta = x_p - v0 (d), M delta (d^2
    products, d (d - 1) sums), lambda_0 (d differences) and the containment
    test (d + 1 compares)."""
    per_eval = dim + dim * dim + dim * (dim - 1) + dim + (dim + 1)
    return n * 2 * dim + sum_path * per_eval
# useful FLOPs of the grid predictor per ASG cell (2-D): conv1 2*18*32, conv2-4
# 3 * 2*288*32, fc1 2*32*256, fc2 2*256*2
CNN_FLOP_PER_CELL_2D = 2 * (18 * 32 + 3 * 288 * 32 + 32 * 256 + 256 * 2)


# useful FLOPs of the classifier predictor per particle: conv1 2*W^d*(d*3^d)*32,
# conv2 2*W^d*(32*3^d)*32, offset branch 2*(d*256 + 256*256), fusion
# 2*(32*(W/2)^d + 256)*512, logits 2*512*W^d (W = 9 in 2-D, 7 in 3-D)
def cls_flops_per_particle(dim):
    W = 9 if dim == 2 else 7
    P, taps = W ** dim, 3 ** dim
    pooled = 32 * (W // 2) ** dim
    return 2 * (P * dim * taps * 32 + P * 32 * taps * 32 + dim * 256 + 256 * 256
                + (pooled + 256) * 512 + 512 * P)


def rank_info():
    r = int(os.environ.get("RANK", "0"))
    w = int(os.environ.get("WORLD_SIZE", "1"))
    lr = int(os.environ.get("LOCAL_RANK", str(r)))
    return r, w, lr


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    return 6800.0, 1900.0, "fallback"


def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2412_18379_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


WALK_SOURCES = ("walk.cu", "walk_common.cuh")
CNN_SOURCES = ("cnn_tc.cu", "tc_common.cuh")
CNN3D_SOURCES = ("cnn3d_tc.cu", "tc_common.cuh")


def ncu_traffic(profile, sources):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on
    the current source; else None."""
    prof = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(prof):
        return None
    vals = {}
    for line in open(prof):
        if ":" in line and line.startswith("- "):
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("source_sha256_16") != source_sha(sources):
        return None
    try:
        return float(vals["dram_bytes_per_full_launch"])
    except (KeyError, ValueError):
        return None


def nvtx_push(name):
    """Open an NVTX range if this PyTorch build has NVTX; True if opened."""
    import torch
    try:
        torch.cuda.nvtx.range_push(name)
        return True
    except (AttributeError, RuntimeError):
        return False


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

    result = None

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
        self.result = {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx,
                       "reasons": sorted(reasons), "samples": len(sm)}
        return self.result


def particle_set(case, kind):
    """(x, u, start) of the particles: one per mesh node (start None: the
    node's element), or one per (element, node) pair starting from the element."""
    from workloads import element_node_particles
    if kind == "element-nodes":
        return element_node_particles(case)
    return case.x, case.u, None


def shard_particles(px, pu, pstart, node_starts, rank, world):
    """This rank's contiguous slice [lo, hi) of one particle batch
    (shard_range); particles that are mesh nodes get their node's element as
    an explicit start. Returns (x, u, start, (lo, hi))."""
    from paper_2412_18379_gb300.shard import shard_range
    lo, hi = shard_range(px.shape[0], rank, world)
    st = pstart if pstart is not None else node_starts
    return (np.ascontiguousarray(px[lo:hi]), np.ascontiguousarray(pu[lo:hi]),
            np.ascontiguousarray(st[lo:hi], dtype=np.int32), (lo, hi))


def cpu_oracle_rate(case, sample_n, seed=0, particles="nodes", threads=1, om=None):
    """The oracle as it stands (plain C through ctypes; its particle loops on
    `threads` OpenMP threads) on a bounded sample of the workload's particles:
    departure point, Algorithm 1 walk from the plain start, exact host.
    Returns (particles/s, seconds, threads used)."""
    import oracle
    if om is None:
        om = oracle.Mesh(case.xyz, case.conn)
    px, pu, pstart = particle_set(case, particles)
    rng = np.random.default_rng(seed)
    idx = np.sort(rng.choice(px.shape[0], size=min(sample_n, px.shape[0]), replace=False))
    start = om.node_elem[idx] if pstart is None else pstart[idx]
    used = oracle.set_threads(threads)
    try:
        t0 = time.perf_counter()
        om.track(px[idx], pu[idx], case.dt, start=start, mode="sns")
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return idx.size / dt, dt, used


def run_reference(args):
    """The reference arm: the oracle timed on every host core of the box (no
    reference code exists besides the paper), each step a bounded sample of
    the workload."""
    r, w, _ = rank_info()
    if r != 0:
        return 0
    import oracle
    from workloads import make_case
    wl = WORKLOADS[args.workload]
    case = make_case(wl["name"], cfl=args.cfl, n_side=wl["n_side"])
    om = oracle.Mesh(case.xyz, case.conn)
    cores = os.cpu_count() or 1
    sample = args.ref_sample
    times, used = [], 1
    for i in range(args.warmup + args.steps):
        _, dt, used = cpu_oracle_rate(case, sample, seed=i, particles=args.particles,
                                      threads=cores, om=om)
        if i >= args.warmup:
            times.append(dt)
    per_step = float(np.mean(times))
    value = sample / per_step
    line = {
        "impl": "reference", "metric": "particles located/s", "value": value,
        "unit": "particles/s", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl["desc"] + ", CFL %g" % args.cfl,
                   "mode": "sns (the oracle's Algorithm 1 walk + exact host)",
                   "sample_particles": sample},
        "cpu_baseline": {"value": value, "unit": "particles/s", "cores": used, "kind": "oracle",
                         "sample": "%d particles drawn from the workload per step, on %d "
                                   "OpenMP threads" % (sample, used)},
        "e2e": {"value": value, "unit": "particles/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def train_predictor(ctx, mesh, case, n_fields, steps, batch, seed):
    """Pairs from plain SNS on random 8-mode fields of the mesh (CFL 2-16),
    then training on the GPU. Returns a report dict."""
    import torch
    from workloads.fields import fourier_modes_2d, fourier_modes_3d, dt_for_cfl
    from workloads.weights import init_weights
    dim = case.dim
    field = fourier_modes_2d if dim == 2 else fourier_modes_3d
    ctx.load_predictor(dim, init_weights(dim, seed))
    if n_fields == 0:
        return {"pairs": 0, "fields": 0, "note": "untrained predictor (profiling runs)"}
    rng = np.random.default_rng(seed)
    x = torch.from_numpy(case.x).cuda()
    wins, tgts = [], []
    t0 = time.perf_counter()
    for s in range(n_fields):
        u = field(case.xyz, 100 + s)
        dt = dt_for_cfl(u, case.h, rng.uniform(2.0, 16.0))
        ud = torch.from_numpy(u).cuda()
        ctx.grid_velocity(mesh, ud)
        w, t, _ = ctx.training_pairs(mesh, x, ud, dt)
        ctx.track(mesh, x, ud, dt, mode="sns")          # host labels by plain SNS
        wins.append(w)
        tgts.append(t)
    W = torch.cat(wins)
    T = torch.cat(tgts)
    del wins, tgts
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = ctx.train(dim, W, T, batch=batch, steps=steps, lr=1e-3, seed=seed)
    t_train = time.perf_counter() - t0
    n_pairs = int(W.shape[0])
    del W, T
    torch.cuda.empty_cache()
    # held-out 8-mode field at CFL 8: path length with and without the CNN
    u = field(case.xyz, 900)
    dt = dt_for_cfl(u, case.h, 8.0)
    ud = torch.from_numpy(u).cuda()
    a = ctx.track(mesh, x, ud, dt, mode="sns")
    b = ctx.track(mesh, x, ud, dt, mode="cnn")
    torch.cuda.synchronize()
    agree = bool(torch.equal(a["host"], b["host"]))
    return {"pairs": n_pairs, "fields": n_fields, "batch": batch, "steps": steps,
            "pair_generation_s": t_pairs, "train_s": t_train,
            "train_pairs_per_s": steps * batch / t_train, "loss_first": float(losses[0]),
            "loss_last": float(losses[-10:].mean()), "optimizer": "Adam lr 1e-3",
            "heldout_field_cfl8": {
                "mean_path_sns": a["path_len"].double().mean().item(),
                "mean_path_cnn_sns": b["path_len"].double().mean().item(),
                "hosts_identical": agree}}


def classifier_bench(ctx, mesh, case, flush, n_fields, steps, batch, timed, seed, bf16_peak):
    """The paper's classifier predictor (Sec. 2.3, Eq. 7-8) on the headline
    mesh: trained on the GPU on (x_p, label) pairs from plain SNS on random
    8-mode fields (CFL 2-16), then CNN-SNS through it on the headline
    particles (timed with CUDA events, L2 flushed before every step), its
    forward pass timed alone, and the hosts checked against plain SNS."""
    import torch
    from workloads.fields import fourier_modes_2d, fourier_modes_3d, dt_for_cfl
    from workloads.weights import init_classifier
    dim = case.dim
    field = fourier_modes_2d if dim == 2 else fourier_modes_3d
    ctx.load_classifier(dim, init_classifier(dim, seed))
    rng = np.random.default_rng(seed)
    xn = torch.from_numpy(case.xyz).cuda()
    xs, labs = [], []
    t0 = time.perf_counter()
    for s in range(n_fields):
        u = field(case.xyz, 300 + s)
        dt = dt_for_cfl(u, case.h, rng.uniform(2.0, 16.0))
        xp, lab = ctx.classifier_pairs(mesh, xn, torch.from_numpy(u).cuda(), dt)
        xs.append(xp)
        labs.append(lab)
    XP = torch.cat(xs)
    LAB = torch.cat(labs)
    del xs, labs
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = ctx.train_classifier(mesh, XP, LAB, batch=batch, steps=steps, lr=1e-3, seed=seed)
    t_train = time.perf_counter() - t0
    n_pairs = int(XP.shape[0])
    del XP, LAB
    torch.cuda.empty_cache()
    x = torch.from_numpy(case.x).cuda()
    u = torch.from_numpy(case.u).cuda()
    n = x.shape[0]
    stream = torch.cuda.current_stream()
    out = ctx.track_classifier(mesh, x, u, case.dt, start_out=True)     # warm-up
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(timed)]
    l0 = ctx.launches
    marked = nvtx_push("timed_classifier")     # selects these steps for a profiler
    for i in range(timed):
        flush.fill_(i & 0xff)
        ev[i][0].record(stream)
        ctx.track_classifier(mesh, x, u, case.dt, out=out)
        ev[i][1].record(stream)
    if marked:
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    launches = (ctx.launches - l0) // max(1, timed)
    ms = sum(a.elapsed_time(b) for a, b in ev) / timed
    xp = ctx.departure(mesh, x, u, case.dt)
    fa, fb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(1)
    fa.record(stream)
    H = ctx.classifier_forward(mesh, xp)
    fb.record(stream)
    torch.cuda.synchronize()
    fwd_ms = fa.elapsed_time(fb)
    del H
    sns = ctx.track(mesh, x, u, case.dt, mode="sns")
    torch.cuda.synchronize()
    flops = cls_flops_per_particle(dim) * n
    ach = flops / (fwd_ms * 1e-3) / 1e12
    return {"workload": "the headline particles and field", "n_particles": n,
            "window": 9 if dim == 2 else 7, "pairs": n_pairs, "fields": n_fields,
            "batch": batch, "steps": steps, "pair_generation_s": t_pairs, "train_s": t_train,
            "train_pairs_per_s": steps * batch / t_train, "loss_first": float(losses[0]),
            "loss_last": float(losses[-10:].mean()),
            "ms_per_step": ms, "particles_per_s": n / (ms * 1e-3), "launches_per_step": launches,
            "forward_ms": fwd_ms, "walk_and_rest_ms": ms - fwd_ms,
            "mean_path_len": out["path_len"].double().mean().item(),
            "mean_path_len_sns": sns["path_len"].double().mean().item(),
            "start_is_host": (out["start"] == out["host"]).double().mean().item(),
            "hosts_identical_to_sns": bool(torch.equal(out["host"], sns["host"])),
            "roofline": {"bound": "tensor", "achieved": ach, "peak": bf16_peak,
                         "unit": "TFLOP/s", "frac": ach / bf16_peak,
                         "kernel": "classifier forward pass (all its kernels)",
                         "algorithmic_flops_per_launch": flops, "traffic": None}}


def serve_bench(ctx, n_requests, rate, slots, seed, pred_stride, repeats):
    """The serving workload: a Poisson stream of tracking requests over 32
    device-resident meshes (16 triangle meshes of 0.1M-4M elements, jittered
    lattices split along the diagonals, and 16 Kuhn tetrahedral meshes of
    0.5M-6M elements, sizes log-uniform), each with its own resident 8-mode
    velocity field; requests of 1e4-2e6 particles (log-uniform, at most the
    mesh's nodes: a contiguous range of its nodes with their elements as the
    plain starts), CFL U(1, 16), CNN-SNS on the request's mesh and field (the
    2-D and 3-D tensor-core predictors), inputs and result buffers in pinned
    host memory, every request copying its inputs in and its results out.
    p50/p99 are the medians over `repeats` streams of n_requests each."""
    import torch
    from workloads.meshes import lattice_tris_2d, kuhn_3d, serving_mesh_sizes
    from workloads.fields import fourier_modes_2d, fourier_modes_3d
    t0 = time.perf_counter()
    rng = np.random.default_rng(seed)
    entries = []
    n_elems = {2: 0, 3: 0}
    for i, (dim, n_side) in enumerate(serving_mesh_sizes(5)):
        if dim == 2:
            xyz, conn, h = lattice_tris_2d(n_side, 0.25, 500 + i)
            u = fourier_modes_2d(xyz, 700 + i)
        else:
            xyz, conn, h = kuhn_3d(n_side, 0.1, 500 + i)
            u = fourier_modes_3d(xyz, 700 + i)
        m = ctx.upload_mesh(xyz, conn)
        m.set_predictor_grid(pred_stride)
        f = ctx.upload_field(m, u)
        n_elems[dim] += conn.shape[0]
        entries.append(dict(mesh=m, field=f, h=h, n=xyz.shape[0],
                            x=torch.from_numpy(np.ascontiguousarray(xyz)).pin_memory(),
                            u=torch.from_numpy(np.ascontiguousarray(u)).pin_memory(),
                            start=torch.from_numpy(m.node_start_elements()).pin_memory(),
                            umax=float(np.sqrt((u * u).sum(axis=1)).max())))
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    dims = {e["mesh"].id: e["mesh"].dim for e in entries}
    used, _ = ctx.memory_usage()
    # warm-up: one small request per mesh, so that no timed request pays a
    # kernel's first launch
    ctx.serve_start(slots=slots, arena_bytes=4 << 30)
    try:
        warm = [ctx.submit(e["mesh"], e["x"][:10000], e["u"][:10000], 0.5 * e["h"] / e["umax"],
                           start=e["start"][:10000], mode="cnn", field=e["field"])[0]
                for e in entries]
        for t in warm:
            ctx.wait(t, timeout_ms=120000)
    finally:
        ctx.serve_stop()
    # every stream's requests are drawn before it starts, and their results go
    # to slices of one pinned block, as a server reuses its response buffers:
    # the arrival loop does nothing but submit
    plans = []
    for rep in range(repeats):
        plan = []
        for _ in range(n_requests):
            e = entries[rng.integers(len(entries))]
            n = int(np.exp(rng.uniform(np.log(1e4), np.log(min(2e6, e["n"])))))
            off = int(rng.integers(0, e["n"] - n + 1))
            dt = rng.uniform(1.0, 16.0) * e["h"] / e["umax"]
            plan.append((e, n, off, dt, rng.exponential(1.0 / rate)))
        plans.append(plan)
    cap = max(sum(p[1] for p in plan) for plan in plans)
    res = dict(host=torch.empty(cap, dtype=torch.int32, pin_memory=True),
               path_len=torch.empty(cap, dtype=torch.int32, pin_memory=True),
               status=torch.empty(cap, dtype=torch.uint8, pin_memory=True))
    # A server's staging buffers have carried requests before: one DMA pass
    # over every pinned input and result buffer (the first transfer through
    # a page of pinned memory runs far below the link's rate)
    for e in entries:
        for k in ("x", "u", "start"):
            torch.empty(e[k].shape, dtype=e[k].dtype, device="cuda").copy_(e[k], non_blocking=True)
    for v in res.values():
        v.copy_(torch.zeros(v.shape, dtype=v.dtype, device="cuda"), non_blocking=True)
    torch.cuda.synchronize()
    reps = []
    for plan in plans:
        ctx.serve_start(slots=slots, arena_bytes=4 << 30)
        tickets = []
        o = 0
        t_next = time.perf_counter()
        try:
            for e, n, off, dt, gap in plan:
                out = {k: v[o:o + n] for k, v in res.items()}
                o += n
                t_next += gap
                while time.perf_counter() < t_next:
                    pass
                sl = slice(off, off + n)
                t, _ = ctx.submit(e["mesh"], e["x"][sl], e["u"][sl], dt, start=e["start"][sl],
                                  mode="cnn", field=e["field"], out=out)
                tickets.append(t)
            modes = [ctx.wait(t, timeout_ms=120000) for t in tickets]
            r = ctx.serve_report()
            trace = ctx.serve_trace()
        finally:
            ctx.serve_stop()
        r["cnn_sns_share"] = float(np.mean(np.array(modes) == 1))
        # where the time of the slowest requests went: waiting for a slot or
        # arena memory (admit - submit), or running (done - admit)
        wait = np.array([t["admit_ms"] - t["submit_ms"] for t in trace])
        run = np.array([t["done_ms"] - t["admit_ms"] for t in trace])
        r["queue_p99_ms"] = float(np.percentile(wait, 99))
        r["service_p99_ms"] = float(np.percentile(run, 99))
        slow = sorted(trace, key=lambda t: t["done_ms"] - t["submit_ms"])[-4:]
        r["slowest"] = [{"n": t["n"], "dim": dims[t["mesh_id"]], "in_flight": t["in_flight"],
                         "queue_ms": round(t["admit_ms"] - t["submit_ms"], 4),
                         "service_ms": round(t["done_ms"] - t["admit_ms"], 4),
                         "device_ms": {k: round(t[k + "_ms"], 4)
                                       for k in ("h2d", "predict", "walk", "d2h")}}
                        for t in reversed(slow)]
        reps.append(r)
    med = lambda k: float(np.median([r[k] for r in reps]))
    out = {"p50_ms": med("p50_ms"), "p99_ms": med("p99_ms"), "mean_ms": med("mean_ms"),
           "max_ms": med("max_ms"), "particles_per_s": med("particles_per_s"),
           "repeats": [{k: r[k] for k in ("p50_ms", "p99_ms", "max_ms", "particles_per_s",
                                          "completed", "rejected", "max_concurrent", "peak_bytes",
                                          "cnn_sns_share", "queue_p99_ms", "service_p99_ms",
                                          "slowest")} for r in reps],
           "requests_per_repeat": n_requests, "arrival_rate_per_s": rate, "slots": slots,
           "meshes": "16 triangle meshes (%.1fM triangles) + 16 tetrahedral meshes (%.1fM tets), "
                     "each with its own resident 8-mode field" % (n_elems[2] / 1e6, n_elems[3] / 1e6),
           "device_bytes_resident": used, "setup_s": setup_s,
           "includes": "H2D of inputs, CNN-SNS start rule on the request's field, walk, D2H of "
                       "outputs"}
    for e in entries:
        e["mesh"].release()
    return out


class Runner:
    """Times tracking steps of one workload through the library's C ABI.

    A step locates every particle once (cs_track, inputs resident in HBM) on
    the current stream; L2 is flushed by a 256 MB write before every timed
    step, outside the step's events. The timed steps run uninstrumented; the
    per-stage device times (and each roofline's kernel time) come from a
    second, profiled pass over the same steps, whose event records would
    otherwise sit between the kernels of every timed step. An untimed pass
    with start_out then gives the error statistics of Sec. 3.1."""

    def __init__(self, ctx, mesh, case, px, pu, pstart, field, flush, dev, dist, max_over_ranks,
                 units_total=None):
        import torch
        self.torch = torch
        self.ctx, self.mesh, self.case, self.field = ctx, mesh, case, field
        self.flush, self.dev, self.dist, self.max_over_ranks = flush, dev, dist, max_over_ranks
        self.x = torch.from_numpy(px).to(dev)
        self.u = torch.from_numpy(pu).to(dev)
        self.start = None if pstart is None else torch.from_numpy(pstart).to(dev)
        self.n = px.shape[0]
        n = self.n
        self.out = dict(host=torch.empty(n, dtype=torch.int32, device=dev),
                        path_len=torch.empty(n, dtype=torch.int32, device=dev),
                        status=torch.empty(n, dtype=torch.uint8, device=dev))
        self.stream = torch.cuda.current_stream(dev)
        self.world = dist.get_world_size() if dist is not None else 1
        # particles the whole job locates per step: every rank's batch
        # (replicas), or the one batch the ranks share (shards)
        self.units = units_total if units_total is not None else self.world * self.n

    def step(self, mode, dt, out=None, start_out=False):
        return self.ctx.track(self.mesh, self.x, self.u, dt, start=self.start, mode=mode,
                              out=out if out is not None else self.out, stream=self.stream,
                              field=self.field, start_out=start_out)

    def run_steps(self, mode, dt, steps):
        torch = self.torch
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        for i in range(steps):
            self.flush.fill_(i & 0xff)
            ev[i][0].record(self.stream)
            self.step(mode, dt)
            ev[i][1].record(self.stream)
        torch.cuda.synchronize()
        return sum(a.elapsed_time(b) for a, b in ev)

    def measure(self, mode, steps, warmup, sampler=None, dt=None):
        torch, ctx = self.torch, self.ctx
        dt = self.case.dt if dt is None else dt
        for _ in range(warmup):
            self.step(mode, dt)
        torch.cuda.synchronize()
        if self.dist is not None:
            self.dist.barrier()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.start()
        l0 = ctx.launches
        # an NVTX range names the timed steps, so that a profiler can select
        # them (ncu --nvtx --nvtx-include "timed_cnn/")
        marked = nvtx_push("timed_" + mode)
        total = self.run_steps(mode, dt, steps)
        if marked:
            torch.cuda.nvtx.range_pop()
        launches = ctx.launches - l0
        if sampler is not None:
            sampler.stop()
        if self.dist is not None:
            total = self.max_over_ranks(total, device=self.dev)
            self.dist.barrier()
        torch.cuda.synchronize()
        st = ctx.stats(self.out["path_len"], self.out["status"])
        ctx.profile(True)
        ctx.profile_read(reset=True)
        self.run_steps(mode, dt, min(steps, 200))
        prof = ctx.profile_read(reset=True)
        ctx.profile(False)
        # error statistics (untimed): origin error err for every start rule,
        # the predictor's displacement error for CNN-SNS
        o = ctx.track(self.mesh, self.x, self.u, dt, start=self.start, mode=mode,
                      stream=self.stream, field=self.field, start_out=True)
        dhat = None
        if mode == "cnn" and self.field is None:
            # the prediction of this call: the same kernel on the mesh's stored
            # grid velocity, which the call has just resampled from u
            cells = int(np.prod(self.mesh.info()["pred_grid"]))
            dhat = torch.empty((cells, self.case.dim), dtype=torch.float32, device=self.dev)
            ctx.predict(self.mesh, dt, out=dhat)
        err = ctx.track_error(self.mesh, self.x, self.u, dt, o["host"], start=o["start"], dhat=dhat)
        mps = total / steps
        n = self.n
        r = dict(particles_per_s=self.units / (mps * 1e-3), ms_per_step=mps,
                 mean_path_len=st["sum"] / n, max_path_len=st["max"],
                 status_counts=[st["found"], st["outside"], st["fallback"], st["invalid"]],
                 stage_ms_per_step={k: v[1] / max(1, v[0]) for k, v in prof.items() if v[0]},
                 err_mean=err["err_mean"], err_max=err["err_max"])
        if err["n_disp"]:
            r["disp_err_mean"] = err["disp_mean"]
            r["disp_err_max"] = err["disp_max"]
            r["disp_err_mean_cells"] = err["disp_mean"] / float(np.mean(
                (np.array(self.mesh.info()["hi"]) - np.array(self.mesh.info()["lo"]))
                / np.array(self.mesh.info()["pred_grid"])))
        return r, prof, launches


def opt_rates(results):
    """Opt(C) = (C(SNS) - C(CNN-SNS)) / C(SNS) (Sec. 3.1) for the mean path
    length, the step time and the origin error err, and the same rates of
    CNN-SNS against the non-learned ASG-direct start."""
    out = {}
    if "cnn" not in results:
        return out
    c = results["cnn"]
    for base in ("sns", "asg"):
        if base in results:
            b = results[base]
            out["vs_" + base] = {
                "opt_mean_path": (b["mean_path_len"] - c["mean_path_len"]) / b["mean_path_len"],
                "opt_time": (b["ms_per_step"] - c["ms_per_step"]) / b["ms_per_step"],
                "opt_err": ((b["err_mean"] - c["err_mean"]) / b["err_mean"]
                            if b["err_mean"] > 0 else None),
                "speedup": b["ms_per_step"] / c["ms_per_step"]}
    return out


def sweep(ctx, cs, args, rank, dev, dist, max_over_ranks, flush, tg_case, tg_mesh):
    """The configuration list beside the headline: the 1001^2 Taylor-Green
    mesh at CFL 1, 4, 8, 16 and the 101^3 ABC cube at CFL 4, 8, 12, 16, 20,
    each in plain SNS, ASG-direct and CNN-SNS (the 2-D predictor trained for
    the headline; a 3-D one trained here the same way)."""
    from workloads import make_case
    from workloads.fields import dt_for_cfl
    steps = max(10, min(args.steps, 50))
    out = []
    for wname, mesh, case, cfls in (("tg2d", tg_mesh, tg_case, (1, 4, 8, 16)),
                                    ("abc3d", None, None, (4, 8, 12, 16, 20))):
        t0 = time.perf_counter()
        training = None
        if mesh is None:
            case = make_case(wname, cfl=8.0, n_side=WORKLOADS[wname]["n_side"])
            mesh = ctx.upload_mesh(case.xyz, case.conn)
            mesh.set_predictor_grid(args.pred_stride_3d)
            training = train_predictor(ctx, mesh, case, args.train_fields_3d,
                                       args.train_steps_3d, args.train_batch, seed=rank)
        run = Runner(ctx, mesh, case, case.x, case.u, None, None, flush, dev, dist,
                     max_over_ranks)
        rows = []
        for cfl in cfls:
            dt = dt_for_cfl(case.u, case.h, cfl)
            res = {}
            for mode in ("sns", "asg", "cnn"):
                r, _, _ = run.measure(mode, steps, 3, dt=dt)
                res[mode] = {k: r[k] for k in ("ms_per_step", "particles_per_s", "mean_path_len",
                                               "max_path_len", "err_mean", "stage_ms_per_step")
                             if k in r}
                for k in ("disp_err_mean", "disp_err_max"):
                    if k in r:
                        res[mode][k] = r[k]
            rows.append({"cfl": cfl, "modes": res, "opt": opt_rates(res)})
        entry = {"workload": WORKLOADS[wname]["desc"], "n_particles": case.n_particles,
                 "n_elements": case.n_elements,
                 "predictor_grid": mesh.info()["pred_grid"], "steps_per_point": steps,
                 "rows": rows, "seconds": time.perf_counter() - t0}
        if training is not None:
            entry["training"] = training
        out.append(entry)
        if wname != "tg2d":
            mesh.release()
        del run
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="tg2d", choices=sorted(WORKLOADS))
    ap.add_argument("--cfl", type=float, default=8.0)
    ap.add_argument("--mode", default="cnn", choices=["sns", "asg", "cnn"])
    ap.add_argument("--particles", default="nodes", choices=["nodes", "element-nodes"],
                    help="one particle per mesh node, or per (element, node) pair "
                         "((d + 1) n_e particles, each starting from its element)")
    ap.add_argument("--pred-stride", type=int, default=5,
                    help="ASG cells per predictor cell and axis (odd)")
    ap.add_argument("--pred-stride-3d", type=int, default=5,
                    help="the same for the 3-D workload of the sweep")
    ap.add_argument("--train-fields-3d", type=int, default=4)
    ap.add_argument("--train-steps-3d", type=int, default=3000)
    ap.add_argument("--no-sweep", action="store_true",
                    help="skip the CFL sweep over the 2-D and 3-D workloads")
    ap.add_argument("--train-fields", type=int, default=4,
                    help="8-mode fields of training pairs (0: an untrained predictor)")
    ap.add_argument("--train-steps", type=int, default=1000)
    ap.add_argument("--train-batch", type=int, default=4096)
    ap.add_argument("--shard", action="store_true",
                    help="under torchrun: split one particle batch over the ranks "
                         "(shard_range; strong scaling) instead of one batch per rank")
    ap.add_argument("--cls-fields", type=int, default=2,
                    help="random fields whose plain-SNS pairs train the classifier")
    ap.add_argument("--cls-steps", type=int, default=300)
    ap.add_argument("--cls-batch", type=int, default=4096)
    ap.add_argument("--cls-timed", type=int, default=3)
    ap.add_argument("--no-classifier", action="store_true")
    ap.add_argument("--ref-sample", type=int, default=1002001)
    ap.add_argument("--cpu-sample", type=int, default=200000)
    ap.add_argument("--cpu-sample-all", type=int, default=1002001)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=1000.0)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--serve-repeats", type=int, default=3)
    ap.add_argument("--quick", action="store_true",
                    help="time the main mode only (no other modes, e2e or CPU leg); "
                         "used for profiler captures")
    args = ap.parse_args()
    if args.quick:
        args.no_cpu_baseline = True
        args.no_sweep = True
        args.no_classifier = True
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
    from paper_2412_18379_gb300.shard import max_over_ranks
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
    mesh.set_predictor_grid(args.pred_stride)
    info = mesh.info()
    dev = torch.device("cuda", lrank)

    modes = [args.mode] if args.quick else ["sns", "asg", "cnn"]
    training = None
    if "cnn" in modes:
        training = train_predictor(ctx, mesh, case, args.train_fields, args.train_steps,
                                   args.train_batch, seed=rank)

    px, pu, pstart = particle_set(case, args.particles)
    n_total = px.shape[0]
    shard = None
    if args.shard:
        px, pu, pstart, shard = shard_particles(px, pu, pstart, mesh.node_start_elements(),
                                                rank, world)
    field = None
    if pstart is not None and "cnn" in modes:
        # particles that are not the mesh nodes: the predictor reads the
        # resident field of the nodal velocity
        field = ctx.upload_field(mesh, case.u)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    run = Runner(ctx, mesh, case, px, pu, pstart, field, flush, dev, dist, max_over_ranks,
                 units_total=n_total if args.shard else None)

    results = {}
    main_prof = main_launches = None
    clocks = None
    for mode in [args.mode] + [m for m in modes if m != args.mode]:
        steps = args.steps if mode == args.mode else max(3, args.steps // 4)
        sampler = ClockSampler(lrank) if mode == args.mode else None
        r, prof, launches = run.measure(mode, steps, args.warmup, sampler)
        if sampler is not None:
            clocks = sampler.result
            main_prof, main_launches = prof, launches
        results[mode] = r
    ctx.device_status()
    main = results[args.mode]
    n = px.shape[0]
    opt = opt_rates(results)

    # rooflines: the walk (HBM gather) and the grid predictor (tensor cores)
    hbm_peak, bf16_peak, peak_kind = peaks()
    walk_l, walk_ms = main_prof["walk"]
    sum_path = main["mean_path_len"] * n
    alg_bytes = n * (16 * dim + 13) + sum_path * REC_ALG_BYTES[dim]
    walk_roof = {"bound": "hbm", "achieved": alg_bytes / (walk_ms / walk_l * 1e-3) / 1e9,
                 "peak": hbm_peak, "unit": "GB/s", "kernel": "walk_kernel<%d>" % dim,
                 "kernel_ms": walk_ms / walk_l, "algorithmic_bytes_per_launch": alg_bytes,
                 "traffic": ncu_traffic("walk_kernel_%s_%s_ncu.md" % (args.workload, args.mode),
                                        WALK_SOURCES),
                 "peak_source": "%s (MEASURED_PEAKS.json hbm_gbs)" % peak_kind}
    walk_roof["frac"] = walk_roof["achieved"] / hbm_peak
    rooflines = {"walk": walk_roof}
    fp64_ops = walk_fp64_ops(n, dim, sum_path)
    fp64_t = fp64_ops / (walk_ms / walk_l * 1e-3) / 1e12
    rooflines["walk_fp64"] = {
        "bound": "alu", "achieved": fp64_t, "peak": FP64_OPS_PEAK_T, "unit": "TFLOP/s",
        "frac": fp64_t / FP64_OPS_PEAK_T, "kernel": "walk_kernel<%d>" % dim,
        "algorithmic_flops_per_launch": fp64_ops,
        "peak_source": "nominal FP64 1.25 TFLOP/s (an FMA as two flops) = 0.625 T unfused "
                       "operations/s; R1's arithmetic has no FMA",
        "note": "R1's operations counted as if executed in FP64; the walk decides most steps "
                "in certified FP32, so the fraction can pass 1"}
    cnn_l, cnn_ms = main_prof.get("cnn", (0, 0.0))
    if cnn_l and dim == 2:
        flops = CNN_FLOP_PER_CELL_2D * int(np.prod(info["pred_grid"]))
        ach = flops / (cnn_ms / cnn_l * 1e-3) / 1e12
        rooflines["cnn"] = {"bound": "tensor", "achieved": ach, "peak": bf16_peak,
                            "unit": "TFLOP/s", "frac": ach / bf16_peak,
                            "kernel": "cnn2d_tc_kernel", "kernel_ms": cnn_ms / cnn_l,
                            "algorithmic_flops_per_launch": flops,
                            "traffic": ncu_traffic("cnn2d_tc_kernel_tg2d_ncu.md", CNN_SOURCES),
                            "peak_source": "%s (MEASURED_PEAKS.json bf16_tflops, burst)"
                                           % peak_kind}
    dominant = "cnn" if "cnn" in rooflines and cnn_ms > walk_ms else "walk"
    roofline = dict(rooflines[dominant])

    # end to end through the host-pointer entry point (pinned buffers)
    xh = torch.from_numpy(px).pin_memory()
    uh = torch.from_numpy(pu).pin_memory()
    sh = None if pstart is None else torch.from_numpy(pstart).pin_memory()
    hout = dict(host=torch.empty(n, dtype=torch.int32).pin_memory(),
                path_len=torch.empty(n, dtype=torch.int32).pin_memory(),
                status=torch.empty(n, dtype=torch.uint8).pin_memory())
    # The mesh-node workload goes through the nodes call: the particles sit
    # at the uploaded vertices, so a step copies in only u. Other layouts,
    # and the general call for comparison, copy x as well.
    nodes = sh is None and px is case.x and n == mesh.n_vertices

    def host_step(general):
        if general:
            ctx.track_host(mesh, xh, uh, case.dt, start=sh, mode=args.mode, out=hout, field=field)
        else:
            ctx.track_nodes_host(mesh, uh, case.dt, mode=args.mode, out=hout, field=field)

    def time_host(general):
        for _ in range(0 if args.quick else 3):
            host_step(general)
        torch.cuda.synchronize()
        steps = max(3, args.steps // 10) if not args.quick else 1
        t0 = time.perf_counter()
        for _ in range(steps):
            host_step(general)
        sec = (time.perf_counter() - t0) / steps
        if dist is not None:
            sec = max_over_ranks(sec, device=dev)
        return (n_total if args.shard else world * n) / sec

    transfer = ("page-locked host buffers; the call copies the inputs to a device staging "
                "buffer and the results back (cudaMemcpyAsync), then synchronises")
    general = {"value": time_host(True), "unit": "particles/s",
               "h2d_bytes_per_step": n * dim * 16 + (0 if sh is None else n * 4),
               "d2h_bytes_per_step": n * 9, "entry_point": "cs_track_host", "transfer": transfer}
    if nodes:
        e2e = {"value": time_host(False), "unit": "particles/s",
               "h2d_bytes_per_step": n * dim * 8, "d2h_bytes_per_step": n * 9,
               "entry_point": "cs_track_nodes_host",
               "transfer": transfer + "; x is the mesh's resident vertex coordinates",
               "general_call": general}
    else:
        e2e = general

    classifier = None
    if not args.no_classifier and args.particles == "nodes" and not args.shard:
        classifier = classifier_bench(ctx, mesh, case, flush, args.cls_fields, args.cls_steps,
                                      args.cls_batch, args.cls_timed, seed=rank,
                                      bf16_peak=bf16_peak)
        rooflines["classifier"] = classifier["roofline"]
        torch.cuda.empty_cache()

    sweep_rows = None
    if not args.no_sweep and args.particles == "nodes" and args.workload == "tg2d" and not args.shard:
        sweep_rows = sweep(ctx, cs, args, rank, dev, dist, max_over_ranks, flush, case, mesh)

    serving = None
    if not args.quick and args.serve_requests > 0:
        if sweep_rows is None:
            from workloads.weights import init_weights
            ctx.load_predictor(3, init_weights(3, rank))      # untrained: exact, longer walks
        torch.cuda.empty_cache()
        serving = serve_bench(ctx, args.serve_requests, args.serve_rate, args.serve_slots,
                              seed=100 + rank, pred_stride=args.pred_stride,
                              repeats=args.serve_repeats)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        import oracle
        om = oracle.Mesh(case.xyz, case.conn)
        rate1, dt1, _ = cpu_oracle_rate(case, args.cpu_sample, particles=args.particles, om=om)
        cores = os.cpu_count() or 1
        rate_all, dt_all, used = cpu_oracle_rate(case, args.cpu_sample_all,
                                                 particles=args.particles, threads=cores, om=om)
        cpu = {"value": rate_all, "unit": "particles/s", "cores": used, "kind": "oracle",
               "sample": "%d of the %d particles (seeded draw), the oracle's plain SNS: departure "
                         "point + Algorithm 1 walk + exact host, its particle loops on %d OpenMP "
                         "threads, %.2f s" % (min(args.cpu_sample_all, n), n, used, dt_all),
               "single_core": {"value": rate1, "unit": "particles/s", "cores": 1,
                               "sample": "%d particles, %.2f s" % (min(args.cpu_sample, n), dt1)}}

    if rank == 0:
        line = {
            "metric": "particles located/s", "value": main["particles_per_s"],
            "unit": "particles/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"],
            "higher_is_better": True, "scaling": "strong" if args.shard else "weak",
            "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": wl["desc"] + ", CFL %g" % args.cfl,
                       "mode": {"cnn": "CNN-SNS (Algorithm 2)", "sns": "plain SNS",
                                "asg": "ASG-direct"}[args.mode],
                       "particles": ("one per mesh node, from the node's element"
                                     if args.particles == "nodes" else
                                     "one per (element, node) pair, from the element"),
                       "n_particles": n_total, "n_elements": case.n_elements,
                       "asg_grid": info["asg_grid"],
                       "predictor_grid": {"stride": info["pred_stride"],
                                          "cells": info["pred_grid"]},
                       "l2": "flushed by a 256 MB write before every timed step",
                       "parallelism": (("%d shards of one batch of %d particles (shard_range: "
                                         "contiguous slices, this rank [%d, %d)), each rank with "
                                         "its own copy of the mesh, no collective"
                                         % (world, n_total, shard[0], shard[1])) if args.shard else
                                        ("%d replicas: every rank locates its own batch of %d "
                                         "particles against its own copy of the mesh, no "
                                         "collective" % (world, n))) if world > 1 else "1 GPU",
                       "arithmetic": "walk decisions FP64 (certified FP32 filter); predictor "
                                     "BF16 x BF16 -> FP32 on tcgen05"},
            "mean_path_len": main["mean_path_len"], "max_path_len": main["max_path_len"],
            "err_mean": main["err_mean"], "modes": results, "opt": opt,
            "training": training, "classifier": classifier, "serving": serving,
            "sweep": sweep_rows,
            "rooflines": rooflines,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": main_launches, "clocks": clocks,
            "paper_context": "paper (4x Xeon 8269CY, CPU): 95.8% shorter paths, 97.0% less "
                             "time with CNN-SNS on the flow past a sphere (Table 2)",
        }
        print(json.dumps(line))
    mesh.release()
    ctx.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
