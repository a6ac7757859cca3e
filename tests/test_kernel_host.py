"""CPU parity of the advection kernel's device code: csrc/tracer.cuh's
advect_node, compiled with g++ (tests/cuda_host_shim.h stands in for the CUDA
built-ins) and run node by node on the host (tests/kernel_host_check.cpp),
against the oracle on the same seeded inputs, under AddressSanitizer and
UndefinedBehaviorSanitizer.  No GPU: this checks the kernel source's logic
(location, hand-off between macros, tie decisions, P1 / P2 stencils,
interface owners) and its memory accesses wherever a GPU is not available; the
GPU parity tests check the compiled kernels themselves.

The sanitizers stop the program at the first finding.  One check is left out:
the left shift of a negative value in r_floor(double) (tracer.cuh), a known
undefined operation whose fix is queued with the next change of the kernel's
source.

Tolerances as for the GPU: FP64 1e-12, FP32 1e-5 of max |T^n|, node by node."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from _helpers import match_nodes, mesh_for, scalar_for, velocity_for
from paper_2103_02388_gb300 import elm, inputs
from paper_2103_02388_gb300.build import build_library

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2103_02388_gb300")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
TOL = {"fp64": 1e-12, "fp32": 1e-5}


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers not found")
    build_library()
    out = str(tmp_path_factory.mktemp("khc") / "kernel_host_check")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fno-omit-frame-pointer",
           "-fsanitize=address,undefined", "-fno-sanitize=shift-base", "-fno-sanitize-recover=all",
           "-I", os.path.join(CUDA, "include"), "-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc"),
           "-include", os.path.join(ROOT, "tests", "cuda_host_shim.h"),
           os.path.join(ROOT, "tests", "kernel_host_check.cpp"), "-o", out,
           "-L", PKG, "-lelm", "-Wl,-rpath," + PKG, "-L", os.path.join(CUDA, "lib64"), "-lcudart"]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stdout + b.stderr
    return out


def _host_step(exe, tmp, v, m, level, precision, order, T, u_old, u_new, dt, n_sub):
    """One step through the host build of the kernel code; T, u in the
    oracle's unique node order; returns T^{n+1} in that order."""
    om_coords = oracle.OracleMesh(v, m, level, order=order).coords
    gm = elm.Mesh(v, m, level, precision, order=order, host_only=True)
    perm = match_nodes(om_coords, gm.unique_coords())
    umap = gm.unique_map()

    def storage(a):
        g = np.empty_like(a)
        g[perm] = a
        return np.ascontiguousarray(g[umap], dtype=np.float64)

    dim = v.shape[1]
    hd = np.array([dim, v.shape[0], m.shape[0], level, 0 if precision == "fp64" else 1, order,
                   1 if u_new is None else 0, n_sub], dtype=np.int64)
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    with open(fin, "wb") as f:
        for a in (hd, np.array([dt], np.float64), np.ascontiguousarray(v, np.float64),
                  np.ascontiguousarray(m, np.int64), storage(u_old), storage(u_old if u_new is None else u_new),
                  storage(T)):
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = np.fromfile(fout, dtype=np.float64)
    uniq = np.empty(gm.n_unique)
    uniq[umap] = out
    assert np.array_equal(uniq[umap], out), "storage copies of a node disagree"
    return uniq[perm]


def _rounded(a, precision):
    return a.astype(np.float32).astype(np.float64) if precision == "fp32" else a


@pytest.mark.parametrize("mesh,level,vel,scal,cfl,n_sub,precision,order", [
    ("square", 4, "rotation", "gauss", None, 1, "fp64", 2),
    ("square", 3, "rotation", "quadratic", 3.0, 3, "fp64", 2),
    ("square_block", 2, "fourier", "gauss", 6.0, 2, "fp64", 2),
    ("cube", 3, "cellular", "slotted", 4.0, 2, "fp64", 2),
    ("cube", 2, "rotation", "gauss", 5.0, 2, "fp64", 2),       # leaves the cube: clamping
    ("cube_block", 1, "fourier", "gauss", 8.0, 2, "fp64", 2),  # 48 perturbed macros: walk
    ("cube", 4, "fourier", "gauss", 4.0, 1, "fp64", 1),        # P1
    ("square", 5, "fourier", "gauss", 4.0, 2, "fp32", 2),
    ("cube", 3, "cellular", "slotted", 8.0, 2, "fp32", 2),
    ("cube_block", 1, "fourier", "gauss", 8.0, 1, "fp32", 2),
    ("cube", 4, "cellular", "gauss", 4.0, 1, "fp32", 1),       # P1
])
def test_kernel_code_matches_oracle(exe, tmp_path, mesh, level, vel, scal, cfl, n_sub, precision, order):
    v, m = mesh_for(mesh)
    om = oracle.OracleMesh(v, m, level, order=order)
    u = _rounded(velocity_for(vel, om.coords), precision)
    T = _rounded(scalar_for(scal, om.coords), precision)
    dt = 1 / 200 if cfl is None else inputs.dt_for_cfl(cfl, level, u)
    got = _host_step(exe, tmp_path, v, m, level, precision, order, T, u, None, dt, n_sub)
    ref = om.advect(T, u, dt, n_sub)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(T).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kernel_code_time_dependent(exe, tmp_path, precision):
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, 3)
    u0 = _rounded(inputs.cellular_flow(om.coords), precision)
    u1 = _rounded(inputs.random_fourier(om.coords, seed=4), precision)
    T = _rounded(scalar_for("gauss", om.coords), precision)
    dt = inputs.dt_for_cfl(3.0, 3, u1)
    got = _host_step(exe, tmp_path, v, m, 3, precision, 2, T, u0, u1, dt, 3)
    ref = om.advect(T, u0, dt, 3, u_new=u1)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(T).max()
