"""The benchmark's JSON contract on the CPU: the reference arm (the oracle on the host cores)
prints one line with the keys the GPU arm prints, on the same workload config."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload",
                          "ising_L8_h4_m1", "--steps", "2", "--warmup", "3"], cwd=ROOT,
                         capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    line = [x for x in out.stdout.splitlines() if x.startswith("{")][-1]
    d = json.loads(line)
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
                "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    c = d["config"]
    assert c["workload"] == "ising_L8_h4_m1" and c["L"] == 8 and c["windows"] == 4
    assert d["step_work"] == {"rounds": 1, "attempts": 4 * 1 * 10_000}
    # a step is one round on one core; the cores run in parallel, so the steps reported are
    # cores x rounds and ms_per_step x steps is the timed wall time of the sample
    cores = d["cpu_baseline"]["cores"]
    assert d["steps"] == cores * max(1, -(-2 // cores))
    wall = float(d["cpu_baseline"]["sample"].rsplit(", ", 1)[1].split(" s")[0])
    assert abs(d["ms_per_step"] * d["steps"] / 1e3 - wall) <= 0.05 + 0.01 * wall
    assert abs(d["value"] - d["steps"] * 40_000 / (d["ms_per_step"] * d["steps"] / 1e3)) < 1e-6 * d["value"]


def test_workload_config_matches_between_arms():
    sys.path.insert(0, ROOT)
    import argparse
    import bench
    args = argparse.Namespace(workload="ising_L64_h32_m16", lnf_init=1.0)
    c = bench.workload_config(args, bench.WORKLOADS["ising_L64_h32_m16"], 1)
    assert c["walkers"] == 512 and c["interval"] == 10_000
    assert c["parallelism"] == "1gpu"
    assert bench.workload_config(args, bench.WORKLOADS["ising_L64_h32_m16"], 4)["parallelism"] == "replicas4"


def test_recorded_traffic_only_for_the_profiled_kernel(tmp_path, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    prof = tmp_path / "profiles"
    prof.mkdir()
    (prof / "k_move_w.md").write_text(
        f"- traffic_bytes_per_launch: 1234\n- kernel_source_digest: {bench.kernel_source_digest()}\n")
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    # the kernel sources are read from ROOT too: point them back at the repository
    monkeypatch.setattr(bench, "KERNEL_SOURCES", [os.path.join(ROOT, f) for f in bench.KERNEL_SOURCES])
    assert bench.recorded_traffic("w") == 1234
    (prof / "k_move_w.md").write_text("- traffic_bytes_per_launch: 1234\n- kernel_source_digest: 0\n")
    assert bench.recorded_traffic("w") is None
    assert bench.recorded_traffic("absent") is None
