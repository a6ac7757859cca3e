"""CPU check of the adjoint's FP32 scaled rounding (csrc/scaled_round.cuh):
integer shifts of the significand must give llrint(ldexp(double(c), k)) for
every finite FP32 c within the slot-scale range (tests/scaled_round_check.cu);
no GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2103_02388_gb300", "csrc")


def test_scaled_round_matches_llrint_ldexp(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "scaled_round_check")
    b = subprocess.run([nvcc, "-O2", "-std=c++17", "-I", CSRC, os.path.join(ROOT, "tests", "scaled_round_check.cu"),
                        "-o", exe], capture_output=True, text=True)
    assert b.returncode == 0, b.stdout + b.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and "all ok" in r.stdout, r.stdout + r.stderr
