"""The library's internal host helpers, compiled with the host compiler
alone (no GPU): the overlap test behind the aliasing checks of every entry
point that writes a vector, and the graph-cache key's separation of solve
variants."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA_INC = "/usr/local/cuda/include"


def test_internal_host_helpers(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("needs g++ and the CUDA headers")
    exe = tmp_path / "host_helpers_check"
    cmd = [cxx, "-std=c++17", "-O1", "-I", CUDA_INC, "-I", os.path.join(ROOT, "paper_2112_11880_gb300", "csrc"),
           "-I", os.path.join(ROOT, "include"), os.path.join(HERE, "host_helpers_check.cpp"), "-o", str(exe)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=30)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
