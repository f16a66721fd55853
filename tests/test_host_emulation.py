"""The library's per-site sweep bodies run on the host (no GPU): even-odd
against whole-lattice sweeps, split-field against FP32 sweeps, the split
step's element mapping, and double-float against FP64 sweeps.  The checks
live in tests/host_emu/kernel_bodies_check.cu, compiled here for the CPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1808_05506_gb300", "csrc")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    return None


def test_kernel_bodies_on_the_host(tmp_path):
    nvcc = _nvcc()
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "kernel_bodies_check")
    src = [os.path.join(HERE, "host_emu", "kernel_bodies_check.cu"), os.path.join(CSRC, "dirac_eo.cu"),
           os.path.join(CSRC, "apply_brillouin.cu")]
    cmd = [nvcc, "-O1", "-std=c++17", "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           "-o", exe] + src
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-3000:]
    r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:]
    assert "all checks hold" in r.stdout
