"""Host-side planning arithmetic of the CUDA path, checked on the CPU: the
stream-K unit ranges (coverage, piece counts, partial-sum slots) and the
split chooser (`csrc/nb_internal.cuh`).  Compiles `tests/host/plan_check.cu`
with nvcc; the program makes no CUDA call, so no GPU is needed."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _nvcc():
    for c in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_plan_arithmetic(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not available")
    exe = str(tmp_path / "plan_check")
    src = os.path.join(HERE, "host", "plan_check.cu")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-gencode", "arch=compute_103a,code=sm_103a",
                    src, "-o", exe], check=True, capture_output=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok"), r.stdout
