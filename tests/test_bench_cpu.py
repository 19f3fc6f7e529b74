"""CPU checks of bench.py: the reference arm (the FP64 oracle on the host cores) prints one JSON line with
the keys of the benchmark contract, on the same workload description as the GPU arm; a committed traffic
figure is used only for the kernel source and the kind of launch it was taken on."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--walls", "64", "--year-steps", "120",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 2 and line["warmup"] == 1
    assert line["value"] > 0 and line["higher_is_better"] is True and line["dtype"] == "f64"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["cpu_baseline"]["value"] == line["value"] and "sample" in line["cpu_baseline"]
    assert line["e2e"]["value"] == line["value"] and line["e2e"]["unit"] == line["unit"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    # the same workload description the GPU arm prints for these sizes
    from paper_1703_10119_gb300 import workloads as wk
    wl = wk.wall_batch(n_walls=64, n_steps=120)
    want = bench.batch_config(wl, 120)
    for k, v in want.items():
        assert line["config"][k] == v, k


def test_traffic_is_used_only_for_a_matching_capture(tmp_path):
    src = bench.kernel_source_hash(bench.KERNEL_SOURCES_2D)
    p = tmp_path / "t.json"
    p.write_text(json.dumps({"kernel_source_sha": src, "dram_bytes_per_launch": 123}))
    assert bench.measured_traffic(str(p), bench.KERNEL_SOURCES_2D) == 123
    p.write_text(json.dumps({"kernel_source_sha": src, "dram_bytes_per_launch": 123, "launch_start_step": 52560}))
    assert bench.measured_traffic(str(p), bench.KERNEL_SOURCES_2D) is None
    p.write_text(json.dumps({"kernel_source_sha": "0" * 16, "dram_bytes_per_launch": 123}))
    assert bench.measured_traffic(str(p), bench.KERNEL_SOURCES_2D) is None
    p.write_text("not json")
    assert bench.measured_traffic(str(p), bench.KERNEL_SOURCES_2D) is None
