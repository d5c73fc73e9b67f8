"""Host-side checks of internal helpers of the CUDA engine, compiled by nvcc
into a host program that makes no CUDA call (no GPU needed): the
per-device set-up record (a second GPU in the same process gets its own
shared-memory opt-in and cluster count) and the triangular tile numbering."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2409_01712_gb300", "csrc")


def _nvcc():
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    return None


def test_per_device_record_and_tile_numbering(tmp_path):
    nvcc = _nvcc()
    if not nvcc:
        pytest.skip("needs nvcc")
    exe = tmp_path / "per_device_check"
    src = os.path.join(ROOT, "tests", "host", "per_device_check.cpp")
    subprocess.run([nvcc, "-x", "cu", "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    "-I", CSRC, src, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, (r.returncode, r.stdout, r.stderr)
    assert r.stdout.strip() == "ok"
