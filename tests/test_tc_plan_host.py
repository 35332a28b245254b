"""Host logic of the tensor-core block matvec (CPU): the unit plan and
schedule (coverage, unit order, load balance) and the formulation behind the
kernel (interleaved complex rows, two real column forms per complex input,
power-of-two scaling, FP16 hi + lo split with three products, FP32 sums),
emulated on a ragged block against the exact complex products."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_tc_plan_and_formulation(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "tc_plan"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_10907_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_src", "tc_plan.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
