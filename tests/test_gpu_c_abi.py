"""The library driven from plain C (tests/c_abi_example.c): no Python or torch on the path.
Built with nvcc against include/lbm.h and liblbm_gb300.so, run, and its own checks
(invariants, phi budget, bounds) must pass."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c_caller(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    libdir = os.path.join(ROOT, "paper_2409_03401_gb300")
    assert os.path.exists(os.path.join(libdir, "liblbm_gb300.so")), "build the library first"
    exe = str(tmp_path / "c_abi_example")
    build = subprocess.run([nvcc, "-O2", "-o", exe, os.path.join(ROOT, "tests", "c_abi_example.c"),
                            "-I", os.path.join(ROOT, "include"), "-L", libdir, "-llbm_gb300",
                            "-Xlinker", f"-rpath={libdir}"], capture_output=True, text=True)
    assert build.returncode == 0, build.stderr
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    print(run.stdout, run.stderr)
    assert run.returncode == 0, run.stderr
    assert "c_abi_example ok" in run.stdout
