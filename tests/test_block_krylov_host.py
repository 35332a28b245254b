"""Host logic of block flexible GMRES (CPU): the deflating Cholesky
normalisation of a block of new Krylov vectors (a dependent column is
dropped, the kept columns are orthonormal and W = V R) and the progressive
Householder QR of the block Hessenberg matrix (the coefficients solve the
least-squares problem of every right-hand side, checked through the normal
equations, and the residual estimates equal the true residual norms), with
the zero rows and columns that a deflated direction produces."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_block_lsq_and_deflating_cholesky(tmp_path):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("needs g++")
    exe = tmp_path / "block_lsq"
    subprocess.run([cxx, "-O2", "-std=c++17", "-pthread", "-I", os.path.join(ROOT, "paper_2502_10907_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "host_src", "block_lsq.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
