"""CPU check of the diffusion operator's host-side set-up: the node-centred
stencil weights of the macro interiors, the interior node lists and the
assembled shared-face rows against a direct element-by-element assembly of
scale (M + alpha A) x (tests/diffusion_host_check.cu; unit cube and square,
levels 0-4, P1 and P2, and a perturbed 48-macro block).  The check program
includes diffusion.cu and links the in-tree library for mesh creation
(host-only meshes); no GPU."""
import os
import shutil
import subprocess

import pytest

from paper_2103_02388_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2103_02388_gb300")


def test_diffusion_host_structures(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    build_library()
    exe = str(tmp_path / "diffusion_host_check")
    cmd = [nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O1", "-std=c++17",
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc"),
           os.path.join(ROOT, "tests", "diffusion_host_check.cu"), "-o", exe,
           "-L", PKG, "-lelm", "-Xlinker", "-rpath=" + PKG]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stdout + b.stderr
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and "all ok" in r.stdout, r.stdout + r.stderr
