"""Host logic of the inner FGMRES (CPU): the complex Givens QR of the
Hessenberg matrix that the recycled second cycle builds its space from.
H-bar = Q R with Q = G_0^H ... G_{k-1}^H [I; 0] and R the rotated columns
must reproduce the columns fed in and Q must have orthonormal columns."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_hessenberg_qr_reproduces_columns(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "krylov_qr"
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", os.path.join(ROOT, "paper_2502_10907_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_src", "krylov_qr.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
