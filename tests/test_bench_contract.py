"""The benchmark's reference arm (the CPU oracle) runs without a GPU; its
JSON line must carry the keys the benchmark contract names."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "0"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600, check=True).stdout
    line = json.loads(out.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["value"] > 0 and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    import bench

    assert line["config"] == bench.workload_config(bench.BUDGET)  # the GPU arm's workload


def test_reference_arm_other_ranks_exit_quietly():
    """Under torchrun only rank 0 runs the reference arm and prints its line;
    the other ranks exit 0 without work or output."""
    env = dict(os.environ, RANK="1", LOCAL_RANK="1", WORLD_SIZE="2")
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--gpus", "2", "--steps", "1",
                        "--warmup", "0"], cwd=ROOT, capture_output=True, text=True, timeout=600, env=env)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_profile_figures_follow_the_kernel_source(tmp_path):
    """A figure from an ncu summary is used only while the summary names the
    current kernel source's hash; otherwise the bench reports null."""
    import hashlib

    import bench

    src = os.path.join(ROOT, "paper_1804_02867_gb300", "csrc", "efm_kernels.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    f = tmp_path / "summary.md"
    f.write_text(f"kernel_source_sha256_16: {sha}\ndram_to_algorithmic_ratio: 1.25\n")
    assert bench.profile_figure(str(f), "dram_to_algorithmic_ratio") == 1.25
    assert bench.profile_figure(str(f), "dram_bytes_per_launch_full_scale") is None
    f.write_text("kernel_source_sha256_16: 0123456789abcdef\ndram_to_algorithmic_ratio: 1.25\n")
    assert bench.profile_figure(str(f), "dram_to_algorithmic_ratio") is None
    assert bench.profile_figure(str(tmp_path / "absent.md"), "dram_to_algorithmic_ratio") is None
