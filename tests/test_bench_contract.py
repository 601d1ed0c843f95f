"""The benchmark's reference arm (the FP64 oracle) keeps the JSON-line contract (CPU only): one
line with the metric, the timing fields, the workload config, the CPU baseline and an end-to-end
entry without host-device bytes; under several ranks only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _run(env_extra, *args):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "d2_N1024_k16", *args], capture_output=True, text=True, env=env, cwd=ROOT,
                       timeout=300)
    return r.returncode, [ln for ln in r.stdout.splitlines() if ln.startswith("{")]


def test_reference_arm_prints_one_contract_line():
    rc, lines = _run({}, "--steps", "2", "--warmup", "3")
    assert rc == 0 and len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 3 and d["value"] > 0
    assert d["higher_is_better"] is True and d["config"]["workload"] == "d2_N1024_k16"
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["unit"] == d["unit"]
    e2e = d["e2e"]
    assert e2e["value"] == d["value"] and e2e["unit"] == d["unit"]
    assert e2e["h2d_bytes_per_step"] == 0 and e2e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_exit_quietly():
    rc, lines = _run({"RANK": "1", "WORLD_SIZE": "2"}, "--steps", "1", "--warmup", "3", "--gpus", "2")
    assert rc == 0 and lines == []


def test_cpu_baseline_reports_one_core_and_all_cores():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--cpu-baseline-only", "--workload",
                        "d2_N1024_k16", "--cpu-seconds", "0.5", "--cpu-all-cores"], capture_output=True, text=True,
                       cwd=ROOT, timeout=300)
    assert r.returncode == 0
    d = json.loads(r.stdout.strip().splitlines()[-1])
    assert d["kind"] == "oracle" and d["cores"] == 1 and d["value"] > 0
    ac = d["all_cores"]
    assert ac["cores"] >= 1 and ac["value"] > 0 and ac["unit"] == d["unit"]
