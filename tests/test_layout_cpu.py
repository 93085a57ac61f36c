"""The host layout builder (lp_host.h: CSC copy, length order, lane-grouped
slices, split rows), compiled into a small host-only program and run on
random matrices and lane policies (tests/host_layout_check.cpp).  No GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(nvcc))


def test_host_layout_builder(tmp_path):
    cuda = _cuda_home()
    inc = os.path.join(cuda, "include")
    if not os.path.exists(os.path.join(inc, "cuda_runtime.h")):
        pytest.skip("CUDA headers not found")
    exe = str(tmp_path / "host_layout_check")
    cmd = ["g++", "-O2", "-std=c++17", "-pthread",
           "-I", os.path.join(ROOT, "paper_2105_12715_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), "-I", inc,
           os.path.join(ROOT, "tests", "host_layout_check.cpp"), "-o", exe,
           "-L", os.path.join(cuda, "lib64"), "-lcudart",
           "-Wl,-rpath," + os.path.join(cuda, "lib64")]
    subprocess.run(cmd, check=True, capture_output=True, timeout=300)
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
