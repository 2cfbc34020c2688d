"""The fused correction MLP's TMEM layout rules, checked on the host from the
kernel's own index functions (tests/native/mlp_tmem_layout.cu, compiled with
nvcc for sm_103a; its main() runs on the CPU and launches nothing)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _nvcc():
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    return None


def test_gelu_blocks_and_runs(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "mlp_tmem_layout")
    src = os.path.join(ROOT, "tests", "native", "mlp_tmem_layout.cu")
    inc = [os.path.join(ROOT, "paper_2606_01009_gb300", "csrc"), os.path.join(ROOT, "include")]
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-std=c++17", "-O1", src, "-o", exe]
    for d in inc:
        cmd += ["-I", d]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    run = subprocess.run([exe], capture_output=True, text=True)
    assert run.returncode == 0, run.stdout[-2000:]
    assert "bad 0" in run.stdout
