"""The incremental Gram-delta mode's copy plan (csrc/inc_plan.cuh), checked
exhaustively on the host for every order m = 36..128 and every cut c: the
ring slots are filled exactly once and the copied units are exactly the
parents' blocks the offspring keeps (tests/inc_plan_check.cu)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_copy_plan_covers_every_cut(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "inc_plan_check")
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2208_14961_gb300", "csrc"),
                    "-o", exe, os.path.join(ROOT, "tests", "inc_plan_check.cu")], check=True, timeout=600)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok: 1944 ")
