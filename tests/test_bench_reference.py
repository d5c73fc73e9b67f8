"""The benchmark's reference arm runs on the host alone (the CPU oracle on a
bounded sample of the headline workload): its JSON line carries the keys the
benchmark contract asks for, and its value agrees with the operation count
over the reported time."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0", "--ref-rows", "256"],
                         capture_output=True, text=True, timeout=600, cwd=ROOT, env=dict(os.environ, WORLD_SIZE="1"))
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in line, key
    assert line["impl"] == "reference" and line["unit"] == "TOp/s" and line["higher_is_better"] is True
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] >= 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # value = operations of the sample / time: N(N+1)M + N^3/3 + 2 N^2 P at N = 256, M = 16384, P = 20
    n, m, p = 256, 16384, 20
    ops = n * (n + 1) * m + n ** 3 / 3.0 + 2.0 * n * n * p
    assert abs(line["value"] - ops / (line["ms_per_step"] / 1e3) / 1e12) <= 1e-9 + 1e-6 * line["value"]
