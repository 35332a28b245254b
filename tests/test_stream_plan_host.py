"""Host logic of the streaming applies (CPU): the unit plan of
stream_plan.h covers every dense entry exactly once, keeps every bulk copy
16-byte aligned inside its row, and lays the tiled copy out unit by unit at
the pitch the kernels assume (compiled with g++, no CUDA)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_stream_plan_invariants(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "stream_plan"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_10907_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_src", "stream_plan.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0 and out.stdout.strip().endswith("ok"), out.stdout + out.stderr
