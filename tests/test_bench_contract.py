"""The bench's reference arm (the FP64 oracle on the host cores) prints one
JSON line with the GPU arm's metric, unit and direction, and the keys the
bench contract names; checked on the small workload, on the CPU."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_line():
    sys.path.insert(0, ROOT)
    import bench
    out = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--workload", "small",
                          "--steps", "1", "--warmup", "0", "--cpu-seconds", "0.3"],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["metric"] == bench.METRIC["small"]
    assert line["unit"] == "active Mpixel-iter/s" and line["higher_is_better"] is True
    assert line["value"] > 0 and line["ms_per_step"] > 0
    for key in ("n_gpus", "steps", "warmup", "scaling", "vs_baseline", "dtype", "data", "config",
                "cpu_baseline", "e2e"):
        assert key in line, key
    import oracle
    cores = oracle.threads() if oracle.has_omp() else 1
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == cores
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["workload"].startswith("cv256")
