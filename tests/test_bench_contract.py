"""The benchmark's reference arm and its JSON line, on the CPU: `bench.py --impl reference`
times the oracle on the same workload and prints one JSON line with the benchmark line's keys."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_the_contract_line():
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--steps", "1", "--warmup", "1",
                        "--ref-runs", "64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["unit"] == "lane-reactions/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0
    assert line["config"]["workload"].startswith("frank_N1024") and "padded" in line["config"]["bound"]


def test_reference_arm_with_the_state_following_bound():
    """--pad 2: the oracle steps whole groups; the line names the bound."""
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--pad", "2", "--steps", "1",
                        "--warmup", "1", "--ref-runs", "64"], cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["config"]["bound"].startswith("2^p per step")


def test_bench_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.algorithmic_ops_per_group_step(19, 11) == 27 * 19 + 6 * 11 + 20 * 6 == 699
    assert bench.algorithmic_ops_per_group_step(19, 11, pad=1) == 680
    assert bench.algorithmic_ops_per_group_step(19, 11, pad=2) == 718
    assert bench.general_ops_per_group_step(19, 11, products=False) == 954
    assert bench.general_ops_per_group_step(19, 11, products=True) == 1473
    assert bench.layout_name(1) == "thread" and bench.layout_name(3) == "thread+warps"
    assert bench.layout_name(1 | 4) == "thread+general incremental" and bench.layout_name(0) == "none"
