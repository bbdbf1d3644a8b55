"""Host-side helpers of bench.py (no GPU): the particle layouts it times, the
ncu-summary lookup behind the roofline's `traffic`, and the CPU baseline."""

import os

import numpy as np
import pytest

import bench
from workloads import make_case


def test_particle_sets():
    c = make_case("rotation2d")
    x, u, start = bench.particle_set(c, "nodes")
    assert x is c.x and u is c.u and start is None
    x, u, start = bench.particle_set(c, "element-nodes")
    assert x.shape == (3 * c.n_elements, 2) and start.shape == (3 * c.n_elements,)
    assert np.array_equal(start[::3], np.arange(c.n_elements))


def _fake_root(tmp_path, source_text, profile_lines):
    root = tmp_path / "root"
    (root / "paper_2412_18379_gb300" / "csrc").mkdir(parents=True)
    (root / "profiles").mkdir()
    (root / "paper_2412_18379_gb300" / "csrc" / "k.cu").write_text(source_text)
    (root / "profiles" / "k_ncu.md").write_text("\n".join(profile_lines) + "\n")
    return root


def test_traffic_only_from_a_summary_of_the_current_source(tmp_path, monkeypatch):
    src = "__global__ void k() {}\n"
    root = _fake_root(tmp_path, src, ["# k"])
    monkeypatch.setattr(bench, "ROOT", str(root))
    sha = bench.source_sha(("k.cu",))
    assert len(sha) == 16
    (root / "profiles" / "k_ncu.md").write_text(
        "# k\n\n- source_sha256_16: %s\n- sources: k.cu\n- dram_bytes_per_full_launch: 1234\n" % sha)
    assert bench.ncu_traffic("k_ncu.md", ("k.cu",)) == 1234.0
    # the kernel changed since the capture: no traffic
    (root / "paper_2412_18379_gb300" / "csrc" / "k.cu").write_text(src + "// edited\n")
    assert bench.ncu_traffic("k_ncu.md", ("k.cu",)) is None
    # no summary, or one without the figure: no traffic
    assert bench.ncu_traffic("missing_ncu.md", ("k.cu",)) is None
    (root / "profiles" / "k_ncu.md").write_text("- source_sha256_16: %s\n"
                                                % bench.source_sha(("k.cu",)))
    assert bench.ncu_traffic("k_ncu.md", ("k.cu",)) is None


def test_committed_summaries_name_their_sources():
    prof = os.path.join(bench.ROOT, "profiles")
    names = [f for f in os.listdir(prof) if f.endswith("_ncu.md")]
    assert names
    for f in names:
        vals = {}
        for line in open(os.path.join(prof, f)):
            if line.startswith("- ") and ":" in line:
                k, v = line[2:].split(":", 1)
                vals[k.strip()] = v.strip()
        assert len(vals["source_sha256_16"]) == 16, f
        for s in vals["sources"].split(","):
            assert os.path.exists(os.path.join(bench.ROOT, "paper_2412_18379_gb300", "csrc", s)), f
        # a summary of one kernel's launch gives its traffic; one of several
        # launches of a general kernel (the training GEMM) gives each table
        if "dram_bytes_per_full_launch" in vals:
            assert float(vals["dram_bytes_per_full_launch"]) > 0, f
        else:
            assert open(os.path.join(prof, f)).read().count("dram__bytes_read.sum") >= 2, f


@pytest.mark.parametrize("particles", ["nodes", "element-nodes"])
def test_cpu_baseline_on_a_sample(particles):
    c = make_case("rotation2d")
    rate, seconds, used = bench.cpu_oracle_rate(c, 500, seed=1, particles=particles)
    assert rate > 0 and seconds > 0 and used == 1
    rate, seconds, used = bench.cpu_oracle_rate(c, 500, seed=1, particles=particles, threads=2)
    assert rate > 0 and seconds > 0 and used in (1, 2)


def test_opt_rates_follow_the_paper_definition():
    """Opt(C) = (C(SNS) - C(CNN-SNS)) / C(SNS), Sec. 3.1; checked on the
    lid-driven cavity values of Table 1 (N_e 8.192e7): mean I_t 11.561 ->
    4.305 gives 62.8%, time 137.233 -> 72.814 s gives 46.9%."""
    res = {"sns": dict(mean_path_len=11.561, ms_per_step=137.233, err_mean=0.0123),
           "cnn": dict(mean_path_len=4.305, ms_per_step=72.814, err_mean=0.0058)}
    o = bench.opt_rates(res)["vs_sns"]
    assert abs(o["opt_mean_path"] - 0.628) < 5e-4
    assert abs(o["opt_time"] - 0.469) < 5e-4
    assert abs(o["opt_err"] - 0.528) < 5e-4
    assert abs(o["speedup"] - 137.233 / 72.814) < 1e-12


def test_shards_cover_the_batch_with_explicit_node_starts():
    """bench.py --shard: the ranks' slices of one batch cover it exactly once,
    in order, and node particles carry their node's element as the start."""
    import bench
    rng = np.random.default_rng(3)
    x = rng.random((1001, 2))
    u = rng.random((1001, 2))
    node = rng.integers(0, 5000, size=1001).astype(np.int32)
    parts = [bench.shard_particles(x, u, None, node, r, 4) for r in range(4)]
    assert [p[3] for p in parts] == [(0, 251), (251, 501), (501, 751), (751, 1001)]
    assert np.array_equal(np.concatenate([p[0] for p in parts]), x)
    assert np.array_equal(np.concatenate([p[1] for p in parts]), u)
    assert np.array_equal(np.concatenate([p[2] for p in parts]), node)
    start = rng.integers(0, 5000, size=1001).astype(np.int32)
    p = bench.shard_particles(x, u, start, node, 1, 4)
    assert np.array_equal(p[2], start[251:501]) and p[2].dtype == np.int32


def test_walk_fp64_operation_count():
    """R1's FP64 operations, counted by hand: 2-D, per evaluation 2
    differences, 4 products, 2 sums, 2 differences for lambda_0, 3 compares
    (13); 3-D, 3 + 9 + 6 + 3 + 4 (25); per particle 2d for the departure."""
    assert bench.walk_fp64_ops(1, 2, 1) == 4 + 13
    assert bench.walk_fp64_ops(10, 3, 25) == 10 * 6 + 25 * 25
    assert bench.walk_fp64_ops(0, 2, 0) == 0
