"""CPU parity of the kernels' device code: csrc/tracer.cuh's advect_node,
csrc/adjoint_kernels.cuh's adjoint kernels, the batched persistent kernel of
csrc/advect.cu and the diffusion operator's kernels of csrc/diffusion.cu (the
stencil and face-row passes, the blended annulus's cell pass and fold, the CG
vector kernels),
compiled with g++ (tests/cuda_host_shim.h stands in for the CUDA built-ins)
and run on the host -- one thread at a time (tests/kernel_host_check.cpp,
tests/adjoint_host_check.cpp), or each block's threads together where the
kernels use barriers, warp shuffles or a shared work counter
(tests/batch_host_check.cpp, tests/diffusion_host_kernels.cpp,
tests/blended_diffusion_host_check.cpp, tests/cg_host_kernels.cpp) -- against the
oracle on the same seeded inputs, under AddressSanitizer and
UndefinedBehaviorSanitizer (and ThreadSanitizer for the block-parallel
kernels).  No GPU: this checks the kernel source's logic
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


def _build(tmp, name, extra=(), tsan=False):
    """Builds tests/<name>.cpp into the directory tmp."""
    gxx = shutil.which("g++")
    out = str(tmp / name)
    if name in ("diffusion_host_kernels", "cg_host_kernels", "blended_diffusion_host_check"):
        # the part of diffusion.cu before the device set-up: kernels and
        # host-built structures, no launches
        with open(os.path.join(PKG, "csrc", "diffusion.cu")) as f:
            src = f.read()
        mark = "elm_status build_diffusion(elm_mesh_s* me"
        assert mark in src, "diffusion.cu no longer has the expected layout"
        with open(str(tmp / "diffusion_front.cuh"), "w") as f:
            f.write("#pragma once\n" + src[:src.index(mark)] + "}  // namespace elm\n")
        extra = list(extra) + ["-I", str(tmp), "-std=c++20", "-DCUDA_HOST_THREADS", "-pthread"]
    if name in ("kernel_host_check", "batch_host_check"):
        # the part of advect.cu before its launch functions: the kernels
        with open(os.path.join(PKG, "csrc", "advect.cu")) as f:
            src = f.read()
        mark = "template <int D, class R, bool STEADY, int P, int MODE>\ncudaError_t launch_k("
        assert mark in src, "advect.cu no longer has the expected layout"
        with open(str(tmp / "advect_front.cuh"), "w") as f:
            f.write("#pragma once\n" + src[:src.index(mark)] + "}  // namespace\n}  // namespace elm\n")
        extra = list(extra) + ["-I", str(tmp)]
        if name == "batch_host_check":
            extra += ["-std=c++20", "-DCUDA_HOST_THREADS", "-pthread"]
    sanitize = (["-fsanitize=thread"] if tsan else
                ["-fsanitize=address,undefined,float-cast-overflow", "-fno-sanitize=shift-base",
                 "-fno-sanitize-recover=all"])
    cmd = [gxx, "-std=c++17", "-O0", "-g", "-fno-omit-frame-pointer", *extra, *sanitize,
           "-I", os.path.join(CUDA, "include"), "-I", os.path.join(ROOT, "include"), "-I", os.path.join(PKG, "csrc"),
           "-I", os.path.join(ROOT, "tests"), "-include", os.path.join(ROOT, "tests", "cuda_host_shim.h"),
           os.path.join(ROOT, "tests", name + ".cpp"), "-o", out,
           "-L", PKG, "-lelm", "-Wl,-rpath," + PKG, "-L", os.path.join(CUDA, "lib64"), "-lcudart"]
    b = subprocess.run(cmd, capture_output=True, text=True)
    assert b.returncode == 0, b.stdout + b.stderr
    return out


PROGRAMS = {"exe": ("kernel_host_check", False), "adj_exe": ("adjoint_host_check", False),
            "diff_exe": ("diffusion_host_kernels", False), "diff_exe_tsan": ("diffusion_host_kernels", True),
            "batch_exe": ("batch_host_check", False), "batch_exe_tsan": ("batch_host_check", True),
            "cg_exe": ("cg_host_kernels", False), "cg_exe_tsan": ("cg_host_kernels", True),
            "blend_diff_exe": ("blended_diffusion_host_check", False),
            "blend_diff_exe_tsan": ("blended_diffusion_host_check", True)}


@pytest.fixture(scope="module")
def programs(tmp_path_factory):
    """All host check programs, built in parallel (each build is one g++ run)."""
    from concurrent.futures import ThreadPoolExecutor
    if shutil.which("g++") is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers not found")
    build_library()
    # the directories first, in this thread (tmp_path_factory is not thread-safe)
    dirs = {k: tmp_path_factory.mktemp(name + ("_tsan" if tsan else "")) for k, (name, tsan) in PROGRAMS.items()}
    with ThreadPoolExecutor(max_workers=len(PROGRAMS)) as ex:
        futs = {k: ex.submit(_build, dirs[k], name, (), tsan) for k, (name, tsan) in PROGRAMS.items()}
        return {k: f.result() for k, f in futs.items()}


@pytest.fixture(scope="module")
def exe(programs):
    return programs["exe"]


@pytest.fixture(scope="module")
def adj_exe(programs):
    return programs["adj_exe"]


@pytest.fixture(scope="module")
def diff_exe(programs):
    return programs["diff_exe"]


@pytest.fixture(scope="module")
def diff_exe_tsan(programs):
    return programs["diff_exe_tsan"]


@pytest.fixture(scope="module")
def batch_exe(programs):
    return programs["batch_exe"]


@pytest.fixture(scope="module")
def batch_exe_tsan(programs):
    return programs["batch_exe_tsan"]


@pytest.fixture(scope="module")
def cg_exe(programs):
    return programs["cg_exe"]


@pytest.fixture(scope="module")
def cg_exe_tsan(programs):
    return programs["cg_exe_tsan"]


@pytest.fixture(scope="module")
def blend_diff_exe(programs):
    return programs["blend_diff_exe"]


@pytest.fixture(scope="module")
def blend_diff_exe_tsan(programs):
    return programs["blend_diff_exe_tsan"]


class HostMesh:
    """The host-only mesh's layout beside the oracle's node order."""

    def __init__(self, v, m, level, precision, order, annulus=None):
        self.v, self.m, self.level, self.precision, self.order = v, m, level, precision, order
        self.annulus = annulus
        om_coords = oracle.OracleMesh(v, m, level, order=order, annulus=annulus).coords
        self.gm = elm.Mesh(v, m, level, precision, order=order, host_only=True, annulus=annulus)
        self.perm = match_nodes(om_coords, self.gm.unique_coords(), **({"tol": 1e-12} if annulus else {}))
        self.umap = self.gm.unique_map()

    def storage(self, a):
        """Unique field (oracle order) -> storage layout, copies everywhere."""
        g = np.empty_like(a)
        g[self.perm] = a
        return np.ascontiguousarray(g[self.umap], dtype=np.float64)

    def unique(self, a):
        """Storage field -> oracle order; checks that all copies of a node agree."""
        a = a.reshape((self.gm.n_nodes,) + (() if a.size == self.gm.n_nodes else (-1,)))
        uniq = np.empty((self.gm.n_unique,) + a.shape[1:])
        uniq[self.umap] = a
        assert np.array_equal(uniq[self.umap], a), "storage copies of a node disagree"
        return uniq[self.perm]


MODE = {"step": 0, "trace": 1, "eval": 2}


def _host_call(exe, tmp, hm, mode, T, u_old, u_new, dt, n_sub, D_in=None):
    """One launch of the host build in `mode`; fields in the oracle's unique
    order, offsets D_in in the storage layout; returns the storage-layout
    result (T, or the offsets for a trace)."""
    dim = hm.v.shape[1]
    hd = np.array([dim, hm.v.shape[0], hm.m.shape[0], hm.level, 0 if hm.precision == "fp64" else 1, hm.order,
                   1 if u_new is None else 0, n_sub, MODE[mode], 0 if D_in is None else 1], dtype=np.int64)
    fin, fout = str(tmp / "in.bin"), str(tmp / "out.bin")
    ann = (0.0, 0.0, 0, 0.0) if hm.annulus is None else hm.annulus
    parts = [hd, np.array([dt, ann[0], ann[1], ann[2], ann[3]], np.float64), np.ascontiguousarray(hm.v, np.float64),
             np.ascontiguousarray(hm.m, np.int64), hm.storage(u_old), hm.storage(u_old if u_new is None else u_new),
             hm.storage(T)]
    if D_in is not None:
        parts.append(np.ascontiguousarray(D_in, np.float64))
    with open(fin, "wb") as f:
        for a in parts:
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    return np.fromfile(fout, dtype=np.float64)


def _host_step(exe, tmp, v, m, level, precision, order, T, u_old, u_new, dt, n_sub):
    """One step through the host build of the kernel code; T, u in the
    oracle's unique node order; returns T^{n+1} in that order."""
    hm = HostMesh(v, m, level, precision, order)
    return hm.unique(_host_call(exe, tmp, hm, "step", T, u_old, u_new, dt, n_sub))


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


@pytest.mark.parametrize("order,level,precision", [(2, 3, "fp64"), (1, 4, "fp64"), (2, 3, "fp32"), (1, 4, "fp32")])
def test_kernel_code_trace_swirl(exe, tmp_path, order, level, precision):
    """The swirling flow of Sec. 3.3 (time-dependent), look-back over 4
    intervals of tau = 0.15 (newest first, offsets carried between intervals
    in the storage layout), then T^0 evaluated at the traced points: offsets
    and field against the oracle's trace continuation.  In FP32 the trace
    mode decides ties in double-float arithmetic."""
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, level, order=order)
    hm = HostMesh(v, m, level, precision, order)
    x = om.coords
    c0 = _rounded(inputs.gaussian(x, (0.35, 0.5, 0.5), 0.1), precision)
    tau = 0.15
    fields = [_rounded(inputs.swirl_3d(x, k * tau), precision) for k in range(5)]
    D = None
    for k in range(len(fields) - 1, 0, -1):
        D = _host_call(exe, tmp_path, hm, "trace", c0, fields[k - 1], fields[k], tau, 2, D_in=D)
    T = hm.unique(_host_call(exe, tmp_path, hm, "eval", c0, fields[0], None, 0.0, 1, D_in=D))
    X = x.copy()
    for k in range(len(fields) - 1, 0, -1):
        X = om.trace(X, fields[k - 1], tau, 2, u_new=fields[k])
    To = om.eval(c0, X)
    dtol = 1e-12 if precision == "fp64" else 2e-5
    assert np.abs((x + hm.unique(D)) - X).max() <= dtol
    assert np.abs(T - To).max() <= (TOL["fp64"] if precision == "fp64" else 2e-4) * np.abs(c0).max()


@pytest.mark.parametrize("level,order,n_sub,speed", [(3, 2, 1, 1.0), (4, 2, 2, 3.0), (4, 1, 1, 2.0), (2, 2, 3, 6.0)])
def test_kernel_code_blended_annulus(exe, tmp_path, level, order, n_sub, speed):
    """The mesh blended onto the annulus r in [0.5, 1.5] (6 sectors, 2D FP64):
    rotation plus a uniform drift, which pushes points across the circles
    (radial clamping), against the oracle's blended step."""
    v, m = inputs.annulus_ring(6, 2)
    ann = (0.5, 1.5, 6, 0.0)
    om = oracle.OracleMesh(v, m, level, order=order, annulus=ann)
    hm = HostMesh(v, m, level, "fp64", order, annulus=ann)
    x = om.coords
    u = speed * (np.stack([-x[:, 1], x[:, 0]], axis=1) + np.array([0.4, -0.25]))
    T = np.exp(-np.sum((x - np.array([0.0, 1.0])) ** 2, axis=1) / 0.05) + 0.2 * x[:, 0]
    got = hm.unique(_host_call(exe, tmp_path, hm, "step", T, u, None, 0.05, n_sub))
    ref = om.advect(T, u, 0.05, n_sub)
    assert np.abs(got - ref).max() <= TOL["fp64"] * np.abs(T).max()


@pytest.mark.parametrize("level,order,dt,n_sub", [(2, 2, 1.6, 1), (3, 1, 1.2, 2), (1, 2, 2.4, 3)])
def test_kernel_code_annulus_across_the_hole(exe, tmp_path, level, order, dt, n_sub):
    """A uniform drift on the annulus with steps longer than the hole's
    diameter: 35-40% of the departure points lie across the hole from their
    node, where the walk meets the inner boundary and the location falls back
    to the search over all macros of the non-convex mesh.  Against the
    oracle's blended step."""
    v, m = inputs.annulus_ring(6, 2)
    ann = (0.5, 1.5, 6, 0.0)
    om = oracle.OracleMesh(v, m, level, order=order, annulus=ann)
    hm = HostMesh(v, m, level, "fp64", order, annulus=ann)
    x = om.coords
    u = np.tile(np.array([1.0, 0.2]), (len(x), 1))
    T = np.exp(-np.sum((x - np.array([-0.8, 0.3])) ** 2, axis=1) / 0.1) + 0.2 * x[:, 0] + 0.1 * x[:, 1] ** 2
    got = hm.unique(_host_call(exe, tmp_path, hm, "step", T, u, None, dt, n_sub))
    ref = om.advect(T, u, dt, n_sub)
    assert np.abs(got - ref).max() <= TOL["fp64"] * np.abs(T).max()


def test_kernel_code_walk_limit_is_a_flag(exe, tmp_path):
    """A step across more macros than the walk limit allows (a 48 x 48 block
    of squares at level 0) ends with the walk-limit flag, not a loop, and no
    sanitizer finding."""
    v, m = inputs.square_block(48)
    hm = HostMesh(v, m, 0, "fp64", 2)
    x = oracle.OracleMesh(v, m, 0).coords
    u = np.tile(np.array([1.0, 0.3]), (len(x), 1))
    with pytest.raises(AssertionError) as e:
        _host_call(exe, tmp_path, hm, "step", np.ones(len(x)), u, None, 0.9, 1)
    msg = str(e.value)
    assert "status flags 1" in msg and "runtime error" not in msg and "AddressSanitizer" not in msg


def test_kernel_code_annulus_non_finite_velocity(exe, tmp_path):
    """A NaN velocity on the annulus: the radial clamp maps the non-finite
    point to a point of the mesh, and the status flag reports it."""
    v, m = inputs.annulus_ring(6, 2)
    ann = (0.5, 1.5, 6, 0.0)
    hm = HostMesh(v, m, 2, "fp64", 2, annulus=ann)
    x = oracle.OracleMesh(v, m, 2, annulus=ann).coords
    u = np.stack([-x[:, 1], x[:, 0]], axis=1)
    u[len(u) // 2] = np.nan
    with pytest.raises(AssertionError) as e:
        _host_call(exe, tmp_path, hm, "step", np.ones(len(x)), u, None, 0.05, 1)
    msg = str(e.value)
    assert "status flags" in msg and "runtime error" not in msg and "AddressSanitizer" not in msg


@pytest.mark.parametrize("direction,level,order", [((1.0, 1.0, 1.0), 3, 2), ((1.0, 1.0, 0.0), 3, 2),
                                                   ((1.0, 1.0, 1.0), 4, 1), ((0.0, 1.0, 1.0), 4, 1)])
def test_kernel_code_departures_on_macro_faces(exe, tmp_path, direction, level, order):
    """A uniform velocity along a Kuhn diagonal keeps the nodes of the planes
    x_i = x_j on them: 10-27% of the departure points lie exactly on interior
    macro faces (in FP32 the location then decides in FP64).  The step equals
    the oracle's at the usual tolerances in both precisions."""
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, level, order=order)
    x = om.coords
    for precision in ("fp64", "fp32"):
        hm = HostMesh(v, m, level, precision, order)
        u = _rounded(np.tile(0.37 * np.array(direction), (len(x), 1)), precision)
        T = _rounded(inputs.random_quadratic(x, seed=5), precision)
        dt = inputs.dt_for_cfl(3.0, level, u)
        got = hm.unique(_host_call(exe, tmp_path, hm, "step", T, u, None, dt, 2))
        ref = om.advect(T, u, dt, 2)
        assert np.abs(got - ref).max() <= TOL[precision] * np.abs(T).max()


@pytest.mark.parametrize("mesh,level,precision,cfl,n_sub", [
    ("cube", 0, "fp64", 40.0, 1), ("cube", 1, "fp64", 12.0, 8), ("square", 0, "fp64", 40.0, 1),
    ("square_block", 2, "fp32", 12.0, 8), ("cube_block", 1, "fp32", 12.0, 8)])
def test_kernel_code_extreme_cfl(exe, tmp_path, mesh, level, precision, cfl, n_sub):
    """Far outside the benchmark regime (CFL 12-40 on the coarsest meshes):
    no sanitizer finding, and T within a bound that allows for the
    conditioning there.  Traces that leave an unstable stagnation point of the
    backward flow (the random Fourier field vanishes at the cube's corners)
    amplify rounding by exp(lambda dt) -- 16 times per interval in the worst
    case -- so two correct implementations that round differently drift
    apart; measured: 1e-10 (FP64) and 1.6e-5 (FP32) of max |T|."""
    v, m = mesh_for(mesh)
    om = oracle.OracleMesh(v, m, level)
    hm = HostMesh(v, m, level, precision, 2)
    u = _rounded(velocity_for("fourier", om.coords), precision)
    T = _rounded(scalar_for("gauss", om.coords), precision)
    dt = inputs.dt_for_cfl(cfl, max(level, 1), u)
    got = hm.unique(_host_call(exe, tmp_path, hm, "step", T, u, None, dt, n_sub))
    ref = om.advect(T, u, dt, n_sub)
    assert np.abs(got - ref).max() <= (1e-8 if precision == "fp64" else 1e-4) * np.abs(T).max()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_kernel_code_non_finite_velocity(exe, tmp_path, precision):
    """A NaN and an infinite velocity value: the status flag (exit 2), and no
    sanitizer finding on the way (conversions, locations of non-finite
    points)."""
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, 2)
    hm = HostMesh(v, m, 2, precision, 2)
    u = velocity_for("fourier", om.coords).copy()
    u[len(u) // 2, 0] = np.nan
    u[len(u) // 3, -1] = np.inf
    T = scalar_for("gauss", om.coords)
    with pytest.raises(AssertionError) as e:
        _host_call(exe, tmp_path, hm, "step", T, u, None, 0.1, 2)
    msg = str(e.value)
    assert "status flags" in msg and "runtime error" not in msg and "AddressSanitizer" not in msg


# ---------------------------------------------------------------------------
# The adjoint (tests/adjoint_host_check.cpp): the cases of the GPU adjoint tests
# at levels 3 (P2) and 4 (P1), the same 17^3 node lattice.

LEVEL = {2: 3, 1: 4}


def _host_adjoint(adj_exe, tmp, v, m, level, precision, order, T, u_old, u_new, g, dt, n_sub):
    """dL/dT^n, dL/du^n, dL/du^{n+1} through the host build of the adjoint
    kernels; inputs and results in the oracle's unique node order, the
    incoming gradient g on owner slots only."""
    om_coords = oracle.OracleMesh(v, m, level, order=order).coords
    gm = elm.Mesh(v, m, level, precision, order=order, host_only=True)
    perm = match_nodes(om_coords, gm.unique_coords())
    umap = gm.unique_map()
    first = np.full(gm.n_unique, -1, np.int64)
    first[umap[::-1]] = np.arange(gm.n_nodes)[::-1]

    def storage(a):
        x = np.empty_like(a)
        x[perm] = a
        return np.ascontiguousarray(x[umap], dtype=np.float64)

    gg = np.empty_like(g)
    gg[perm] = g
    gs = np.zeros(gm.n_nodes)
    gs[first] = gg
    dim = v.shape[1]
    split = u_new is not None
    hd = np.array([dim, v.shape[0], m.shape[0], level, 0 if precision == "fp64" else 1, order,
                   0 if split else 1, n_sub, 1 if split else 0], dtype=np.int64)
    fin, fout = str(tmp / "adj_in.bin"), str(tmp / "adj_out.bin")
    with open(fin, "wb") as f:
        for a in (hd, np.array([dt], np.float64), np.ascontiguousarray(v, np.float64),
                  np.ascontiguousarray(m, np.int64), storage(u_old), storage(u_old if u_new is None else u_new),
                  storage(T), gs):
            f.write(a.tobytes())
    r = subprocess.run([adj_exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    out = np.fromfile(fout, dtype=np.float64)
    n = gm.n_nodes
    gT, gU0, gU1 = out[:n], out[n:n + n * dim].reshape(n, dim), out[n + n * dim:].reshape(n, dim)
    return gT[first][perm], gU0[first][perm], gU1[first][perm]


def _adjoint_fields(x, kind, precision):
    if kind == "linear":
        rng = np.random.default_rng(2)
        u = inputs.linear_field(x, rng.standard_normal((3, 3)), np.full(3, 0.5))
        T = inputs.random_quadratic(x, seed=6)
    else:
        u = inputs.random_fourier(x, seed=9) + 0.2 * inputs.uniform_field(x, [0.31, -0.17, 0.23])
        T = inputs.gaussian(x, (0.45, 0.5, 0.55), 0.15)
    return _rounded(u, precision), _rounded(T, precision)


@pytest.mark.parametrize("precision,n_sub,order", [("fp64", 1, 2), ("fp64", 3, 2), ("fp32", 1, 2),
                                                   ("fp64", 1, 1), ("fp64", 3, 1)])
def test_adjoint_code_transpose(adj_exe, tmp_path, precision, n_sub, order):
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, LEVEL[order], order=order)
    u, T = _adjoint_fields(om.coords, "fourier", precision)
    dt = inputs.dt_for_cfl(4.0, 3, u)
    g = np.random.default_rng(1).standard_normal(om.n_nodes)
    gT, _, _ = _host_adjoint(adj_exe, tmp_path, v, m, LEVEL[order], precision, order, T, u, None, g, dt, n_sub)
    ref = om.advect_transpose(g, u, dt, n_sub)
    assert np.abs(gT - ref).max() <= TOL[precision] * np.abs(ref).max() * 10


@pytest.mark.parametrize("kind,n_sub,order", [("linear", 1, 2), ("linear", 2, 2), ("fourier", 1, 2),
                                              ("fourier", 2, 2), ("fourier", 1, 1)])
def test_adjoint_code_velocity_gradient(adj_exe, tmp_path, kind, n_sub, order):
    """<dL/du, v> against the oracle's forward-mode derivative on 8 random
    directions (L = <g, T^{n+1}>), FP64."""
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, LEVEL[order], order=order)
    u, T = _adjoint_fields(om.coords, kind, "fp64")
    dt = inputs.dt_for_cfl(3.0, 3, u)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(om.n_nodes)
    _, gU, _ = _host_adjoint(adj_exe, tmp_path, v, m, LEVEL[order], "fp64", order, T, u, None, g, dt, n_sub)
    for _ in range(8):
        d = rng.standard_normal(u.shape)
        _, jvp = om.advect_jvp(T, u, d, dt, n_sub)
        assert abs((gU * d).sum() - g @ jvp) <= 1e-9 * (np.abs(g) @ np.abs(jvp) + 1e-30)


@pytest.mark.parametrize("precision,n_sub,order", [("fp64", 1, 2), ("fp64", 2, 2), ("fp32", 1, 2), ("fp64", 1, 1)])
def test_adjoint_code_2d(adj_exe, tmp_path, precision, n_sub, order):
    """The 2D forms: dL/dT^n against the oracle's transpose, and (FP64)
    <dL/du, v> against its forward-mode derivative on 4 random directions."""
    v, m = mesh_for("square")
    level = 5 if order == 2 else 6
    om = oracle.OracleMesh(v, m, level, order=order)
    x = om.coords
    u = _rounded(inputs.random_fourier(x, seed=9) + 0.2 * inputs.uniform_field(x, [0.31, -0.17]), precision)
    T = _rounded(inputs.gaussian(x, (0.45, 0.55), 0.15), precision)
    dt = inputs.dt_for_cfl(4.0, level, u)
    rng = np.random.default_rng(4)
    g = rng.standard_normal(om.n_nodes)
    gT, gU, _ = _host_adjoint(adj_exe, tmp_path, v, m, level, precision, order, T, u, None, g, dt, n_sub)
    ref = om.advect_transpose(g, u, dt, n_sub)
    assert np.abs(gT - ref).max() <= TOL[precision] * np.abs(ref).max() * 10
    if precision == "fp64":
        for _ in range(4):
            d = rng.standard_normal(u.shape)
            _, jvp = om.advect_jvp(T, u, d, dt, n_sub)
            assert abs((gU * d).sum() - g @ jvp) <= 1e-9 * (np.abs(g) @ np.abs(jvp) + 1e-30)


def test_adjoint_code_time_dependent_split(adj_exe, tmp_path):
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, 3)
    u0, T = _adjoint_fields(om.coords, "fourier", "fp64")
    u1 = inputs.random_fourier(om.coords, seed=12) + 0.2 * inputs.uniform_field(om.coords, [-0.21, 0.33, 0.14])
    dt = inputs.dt_for_cfl(3.0, 3, u1)
    rng = np.random.default_rng(8)
    g = rng.standard_normal(om.n_nodes)
    _, gU0, gU1 = _host_adjoint(adj_exe, tmp_path, v, m, 3, "fp64", 2, T, u0, u1, g, dt, 2)
    zero = np.zeros_like(u0)
    for _ in range(4):
        d = rng.standard_normal(u0.shape)
        _, j0 = om.advect_jvp(T, u0, d, dt, 2, u_new=u1, du_new=zero)
        _, j1 = om.advect_jvp(T, u0, zero, dt, 2, u_new=u1, du_new=d)
        assert abs((gU0 * d).sum() - g @ j0) <= 1e-9 * (np.abs(g) @ np.abs(j0) + 1e-30)
        assert abs((gU1 * d).sum() - g @ j1) <= 1e-9 * (np.abs(g) @ np.abs(j1) + 1e-30)


def test_adjoint_code_non_finite_velocity(adj_exe, tmp_path):
    """A NaN velocity value in the adjoint: the status flag (exit 2) and no
    sanitizer finding (scale exponents of non-finite statistics, conversions)."""
    v, m = mesh_for("cube")
    om = oracle.OracleMesh(v, m, 2)
    u, T = _adjoint_fields(om.coords, "fourier", "fp64")
    u = u.copy()
    u[len(u) // 2, 0] = np.nan
    g = np.random.default_rng(1).standard_normal(om.n_nodes)
    with pytest.raises(AssertionError) as e:
        _host_adjoint(adj_exe, tmp_path, v, m, 2, "fp64", 2, T, u, None, g, 0.1, 2)
    msg = str(e.value)
    assert "status flags" in msg and "runtime error" not in msg and "AddressSanitizer" not in msg


def _host_diffusion(exe, tmp, hm, x, alpha, scale, cg):
    v, m = hm.v, hm.m
    hd = np.array([v.shape[1], v.shape[0], m.shape[0], hm.level, 0 if hm.precision == "fp64" else 1, hm.order,
                   int(cg)], dtype=np.int64)
    fin, fout = str(tmp / "d_in.bin"), str(tmp / "d_out.bin")
    with open(fin, "wb") as f:
        for a in (hd, np.array([alpha, scale]), np.ascontiguousarray(v, np.float64), np.ascontiguousarray(m, np.int64),
                  hm.storage(x)):
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ThreadSanitizer" not in r.stderr, r.stderr
    return np.fromfile(fout, dtype=np.float64)


# ---------------------------------------------------------------------------
# The diffusion operator (tests/diffusion_host_kernels.cpp): k_stencil and
# k_face_rows, each block's threads run together (barriers, warp shuffles, the
# last block's completion of the p.q sum), against the oracle's assembled
# mass and stiffness matrices.

@pytest.mark.parametrize("mesh,level,order,precision,cg", [
    ("cube", 2, 2, "fp64", False), ("cube", 3, 1, "fp64", False), ("square", 3, 2, "fp64", False),
    ("cube_block", 1, 2, "fp64", False), ("cube", 2, 2, "fp32", False),
    ("cube", 2, 2, "fp64", True), ("cube_block", 1, 2, "fp64", True), ("square", 3, 1, "fp32", True)])
def test_diffusion_operator_code(diff_exe, tmp_path, mesh, level, order, precision, cg):
    """y = scale (M + alpha A) x at every node off the Dirichlet boundary (and
    y = 0 on it); in the CG form also p.q = x . y over those nodes, summed by
    the kernels' fixed-order reduction."""
    v, m = mesh_for(mesh)
    om = oracle.OracleMesh(v, m, level, order=order)
    hm = HostMesh(v, m, level, precision, order)
    x = _rounded(np.random.default_rng(3).standard_normal(om.n_nodes), precision)
    alpha, scale = 0.37, 1.3
    out = _host_diffusion(diff_exe, tmp_path, hm, x, alpha, scale, cg)
    y, pq = hm.unique(out[:-1]), out[-1]
    M, A = om.assemble()
    ref = scale * (M @ x + alpha * (A @ x))
    bnd = om.boundary()
    tol = 1e-13 if precision == "fp64" else 1e-5
    assert np.abs(y - ref)[~bnd].max() <= tol * np.abs(ref[~bnd]).max()
    assert np.all(y[bnd] == 0)
    if cg:
        pq_ref = x[~bnd] @ ref[~bnd]
        assert abs(pq - pq_ref) <= tol * (np.abs(x[~bnd]) @ np.abs(ref[~bnd]))


@pytest.mark.parametrize("mesh,level,order,precision", [
    ("cube", 2, 2, "fp64"), ("cube_block", 1, 2, "fp64"), ("square", 3, 1, "fp64"), ("cube", 2, 1, "fp32")])
def test_diffusion_operator_code_diagonal(diff_exe, tmp_path, mesh, level, order, precision):
    """The diagonal form of the passes (the Jacobi preconditioner's set-up):
    y = scale diag(M + alpha A) at every node off the Dirichlet boundary, 0 on
    it; x is not read (NaN here)."""
    v, m = mesh_for(mesh)
    om = oracle.OracleMesh(v, m, level, order=order)
    hm = HostMesh(v, m, level, precision, order)
    x = np.full(om.n_nodes, np.nan)
    alpha, scale = 0.37, 1.3
    out = _host_diffusion(diff_exe, tmp_path, hm, x, alpha, scale, 2)
    y = hm.unique(out[:-1])
    M, A = om.assemble()
    ref = scale * (M.diagonal() + alpha * A.diagonal())
    bnd = om.boundary()
    tol = 1e-13 if precision == "fp64" else 1e-6
    assert np.abs(y - ref)[~bnd].max() <= tol * np.abs(ref[~bnd]).max()
    assert np.all(y[bnd] == 0)


@pytest.mark.parametrize("mesh,level,order", [("cube", 2, 2), ("cube_block", 1, 2)])
def test_diffusion_operator_code_has_no_data_race(diff_exe_tsan, tmp_path, mesh, level, order):
    """The same passes in their CG form under ThreadSanitizer: no data race
    between the threads of a block (shared-memory tables, warp exchanges, the
    last block's reduction)."""
    v, m = mesh_for(mesh)
    om = oracle.OracleMesh(v, m, level, order=order)
    hm = HostMesh(v, m, level, "fp64", order)
    x = np.random.default_rng(3).standard_normal(om.n_nodes)
    _host_diffusion(diff_exe_tsan, tmp_path, hm, x, 0.37, 1.3, True)


# ---------------------------------------------------------------------------
# The blended annulus's operator (tests/blended_diffusion_host_check.cpp): the
# per-simplex tables, the cell pass k_apply and its fold k_fold_nodes, each
# block's threads run together, against the oracle's blended mass and
# stiffness matrices (each side with its own 5 x 5 collapsed Gauss rule).

ANNULUS = (0.5, 1.5, 6, 0.0)


def _host_blended_diffusion(exe, tmp, hm, x, alpha, scale, mode):
    v, m = hm.v, hm.m
    hd = np.array([v.shape[0], m.shape[0], hm.level, hm.order, mode], dtype=np.int64)
    fin, fout = str(tmp / "b_in.bin"), str(tmp / "b_out.bin")
    with open(fin, "wb") as f:
        for a in (hd, np.array([alpha, scale, *ANNULUS], np.float64), np.ascontiguousarray(v, np.float64),
                  np.ascontiguousarray(m, np.int64), hm.storage(x)):
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ThreadSanitizer" not in r.stderr, r.stderr
    return np.fromfile(fout, dtype=np.float64)


# The stiffness is where the two sides may differ beyond rounding.  Its
# integrand is rational in the point (the sector parameter of the blending map),
# and the oracle and the tables collapse their 5 x 5 Gauss rules at different
# vertices of the simplex, so each has its own quadrature error.  Measured
# difference of A x, relative to max |A x|: 3.9e-8, 7.9e-10, 1.2e-11, 1.0e-13
# at levels 1-4 (P2); 3.1e-12, 3.0e-14, 4.7e-15 at levels 2-4 (P1).  That is a
# fall of about 60 per level, as a quadrature error should fall, down to
# rounding.  A wrong table entry or a lost contribution would be of order one.
# The mass is exact on both sides (constant Jacobian determinant), so a
# mass-only pass (alpha = 0) is held to rounding.
BLEND_TOL = {(2, 2): 4e-9, (3, 1): 1e-13, (4, 2): 4e-13}


@pytest.mark.parametrize("level,order", [(2, 2), (3, 1), (4, 2)])
@pytest.mark.parametrize("mode", ["mass", "accum", "cg", "diag"])
def test_blended_diffusion_operator_code(blend_diff_exe, tmp_path, level, order, mode):
    """mass / accum: y = scale (M + alpha A) x at every node, boundary included
    (the solver sets the Dirichlet values afterwards; mass: alpha = 0); cg: the
    same with y = 0 on the boundary and p.q = x . y over the other nodes;
    diag: y = scale diag(M + alpha A)."""
    v, m = inputs.annulus_ring(6, 2)
    om = oracle.OracleMesh(v, m, level, order=order, annulus=ANNULUS)
    hm = HostMesh(v, m, level, "fp64", order, annulus=ANNULUS)
    x = np.random.default_rng(5).standard_normal(om.n_nodes)
    alpha, scale = (0.0 if mode == "mass" else 0.37), 1.3
    code = {"mass": 0, "accum": 0, "cg": 1, "diag": 2}[mode]
    out = _host_blended_diffusion(blend_diff_exe, tmp_path, hm, x, alpha, scale, code)
    y, pq = hm.unique(out[:-1]), out[-1]
    M, A = om.assemble()
    bnd = om.boundary()
    assert bnd.any() and not bnd.all()
    if mode == "diag":
        ref = scale * (M.diagonal() + alpha * A.diagonal())
    else:
        ref = scale * (M @ x + alpha * (A @ x))
    tol = 1e-13 if mode == "mass" else BLEND_TOL[(level, order)]
    if mode == "cg":
        assert np.abs(y - ref)[~bnd].max() <= tol * np.abs(ref[~bnd]).max()
        assert np.all(y[bnd] == 0)
        assert abs(pq - x[~bnd] @ ref[~bnd]) <= tol * (np.abs(x[~bnd]) @ np.abs(ref[~bnd]))
    else:
        assert np.abs(y - ref).max() <= tol * np.abs(ref).max()


def test_blended_diffusion_operator_code_has_no_data_race(blend_diff_exe_tsan, tmp_path):
    """The blended passes in their CG form under ThreadSanitizer: no data race
    between the threads of a block (the cell pass's colour accumulators, the
    fold's warp exchanges and the last block's reduction)."""
    v, m = inputs.annulus_ring(6, 2)
    hm = HostMesh(v, m, 2, "fp64", 2, annulus=ANNULUS)
    x = np.random.default_rng(5).standard_normal(hm.gm.n_unique)
    out = _host_blended_diffusion(blend_diff_exe_tsan, tmp_path, hm, x, 0.37, 1.3, 1)
    assert np.all(np.isfinite(out))


# ---------------------------------------------------------------------------
# The batched persistent kernel (tests/batch_host_check.cpp): k_advect_batch,
# each block's threads run together (the shared work-item fetch), over a mix
# of instances.

BATCH = [("square", 3, "rotation", 1.5, 1, True), ("cube", 2, "fourier", 4.0, 2, False),
         ("cube_block", 1, "fourier", 6.0, 1, True), ("square_block", 2, "rotation", 2.0, 2, False),
         ("cube", 3, "cellular", 4.0, 1, True)]


def _batch_inputs(precision):
    out = []
    for k, (mesh, level, vel, cfl, n_sub, steady) in enumerate(BATCH):
        v, m = mesh_for(mesh)
        om = oracle.OracleMesh(v, m, level)
        hm = HostMesh(v, m, level, precision, 2)
        x = om.coords
        u = _rounded(velocity_for(vel, x), precision)
        u1 = u if steady else _rounded(inputs.random_fourier(x, seed=50 + k), precision)
        T = _rounded(scalar_for("gauss", x), precision)
        out.append((om, hm, u, u1, T, inputs.dt_for_cfl(cfl, level, u), n_sub, steady))
    return out


def _host_batch(exe, tmp, precision, inst, chunks_per_item, blocks):
    parts = [np.array([len(inst), 0 if precision == "fp64" else 1, chunks_per_item, blocks], np.int64)]
    for om, hm, u, u1, T, dt, n_sub, steady in inst:
        v, m = hm.v, hm.m
        parts += [np.array([v.shape[1], v.shape[0], m.shape[0], hm.level, int(steady), n_sub], np.int64),
                  np.array([dt]), np.ascontiguousarray(v, np.float64), np.ascontiguousarray(m, np.int64),
                  hm.storage(u), hm.storage(u1), hm.storage(T)]
    fin, fout = str(tmp / "b_in.bin"), str(tmp / "b_out.bin")
    with open(fin, "wb") as f:
        for a in parts:
            f.write(a.tobytes())
    r = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "ThreadSanitizer" not in r.stderr, r.stderr
    out = np.fromfile(fout, dtype=np.float64)
    res, o = [], 0
    for _, hm, *_rest in inst:
        res.append(out[o:o + hm.gm.n_nodes])
        o += hm.gm.n_nodes
    # each result read back in node order (k_gather over the owner copies):
    # every storage copy of a node holds the gathered value
    for g, (_, hm, *_rest) in zip(res, inst):
        gu = out[o:o + hm.gm.n_unique]
        o += hm.gm.n_unique
        assert np.array_equal(gu[hm.umap], g)
    assert o == out.size
    return res


@pytest.mark.parametrize("precision,chunks_per_item,blocks", [("fp64", 1, 3), ("fp64", 4, 2), ("fp32", 2, 5)])
def test_batch_kernel_code(batch_exe, exe, tmp_path, precision, chunks_per_item, blocks):
    """Every instance of the batch equals its own single-instance host step bit
    for bit, and the oracle at the usual tolerance."""
    inst = _batch_inputs(precision)
    got = _host_batch(batch_exe, tmp_path, precision, inst, chunks_per_item, blocks)
    for (om, hm, u, u1, T, dt, n_sub, steady), g in zip(inst, got):
        single = _host_call(exe, tmp_path, hm, "step", T, u, None if steady else u1, dt, n_sub)
        assert np.array_equal(g, single)
        ref = om.advect(T, u, dt, n_sub, u_new=None if steady else u1)
        assert np.abs(hm.unique(g) - ref).max() <= TOL[precision] * np.abs(T).max()


def test_batch_kernel_code_has_no_data_race(batch_exe_tsan, tmp_path):
    """The persistent work fetch (one thread takes the next item from the
    shared counter, the block reads it after a barrier) under ThreadSanitizer,
    with more blocks than the work needs."""
    _host_batch(batch_exe_tsan, tmp_path, "fp64", _batch_inputs("fp64"), 1, 6)


# ---------------------------------------------------------------------------
# The CG solve's vector kernels (tests/cg_host_kernels.cpp), each block's
# threads together, in the order one iteration uses them: every kernel's effect
# against NumPy in the working precision (element-wise results bit for bit:
# the host build does not fuse multiply-adds, and NumPy rounds each operation
# the same way), the sums to their rounding.

def _run_cg(exe, tmp, n, precision, blocks, budget=10, alpha=0.3, stop_rr=1e-30, seed=0):
    rng = np.random.default_rng(seed)
    R = np.float64 if precision == "fp64" else np.float32
    r, q, x, v = (rng.standard_normal(n).astype(R).astype(np.float64) for _ in range(4))
    dinv = (0.5 + rng.random(n)).astype(R).astype(np.float64)
    v[rng.random(n) < 0.05] = 0.0  # zero diagonal entries
    bnd = (rng.random(n) < 0.1).astype(np.uint8)
    act = ((rng.random(n) < 0.75) & (bnd == 0)).astype(np.uint8)
    fin, fout = str(tmp / "cg_in.bin"), str(tmp / "cg_out.bin")
    with open(fin, "wb") as f:
        for a in (np.array([n, 0 if precision == "fp64" else 1, blocks, budget], np.int64),
                  np.array([alpha, stop_rr]), r, dinv, q, x, v, bnd, act):
            f.write(np.ascontiguousarray(a).tobytes())
    res = subprocess.run([exe, fin, fout], capture_output=True, text=True, timeout=600)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "ThreadSanitizer" not in res.stderr, res.stderr
    out = np.fromfile(fout, dtype=np.float64)
    return out, (R, r, dinv, q, x, v, bnd.astype(bool), act.astype(bool), alpha, stop_rr, budget)


@pytest.mark.parametrize("n,precision,blocks", [(1237, "fp64", 3), (5000, "fp32", 5), (64, "fp64", 2)])
def test_cg_vector_kernels_code(cg_exe, tmp_path, n, precision, blocks):
    out, (R, r, dinv, q, x, v, bnd, act, alpha, stop_rr, budget) = _run_cg(cg_exe, tmp_path, n, precision, blocks)
    tol = 1e-13 if precision == "fp64" else 1e-5
    o = 0

    def take(k):
        nonlocal o
        a = out[o:o + k]
        o += k
        return a

    Rv = lambda a: np.asarray(a, dtype=R)  # noqa: E731
    r0 = np.where(bnd, R(0), Rv(r))
    z0 = Rv(dinv) * r0
    assert np.array_equal(take(n), r0) and np.array_equal(take(n), z0) and np.array_equal(take(n), z0)
    rz0 = float(np.dot(r0[act].astype(np.float64), z0[act].astype(np.float64)))
    rr0 = float(np.dot(r0[act].astype(np.float64), r0[act].astype(np.float64)))
    rz, rr, done = take(3)
    assert abs(rz - rz0) <= tol * abs(rz0) and abs(rr - rr0) <= tol * rr0 and done == 0
    al = R(alpha)
    x1 = Rv(x) + al * z0
    r1 = r0 - al * Rv(q)
    z1 = Rv(dinv) * r1
    assert np.array_equal(take(n), x1) and np.array_equal(take(n), r1) and np.array_equal(take(n), z1)
    rz1 = float(np.dot(r1[act].astype(np.float64), z1[act].astype(np.float64)))
    rr1 = float(np.dot(r1[act].astype(np.float64), r1[act].astype(np.float64)))
    rz_new, rr_u, beta, iters, done = take(5)
    assert abs(rz_new - rz1) <= tol * abs(rz1) and abs(rr_u - rr1) <= tol * rr1
    assert abs(beta - rz1 / rz0) <= 4 * tol * abs(rz1 / rz0) and iters == 1 and done == 0
    p1 = z1 + R(beta) * z0
    assert np.array_equal(take(n), p1)
    nrm = take(1)[0]
    assert abs(nrm - float(np.sum(r1[act].astype(np.float64) ** 2))) <= 1e-13 * rr1
    with np.errstate(divide="ignore"):
        d = np.where(bnd | (Rv(v) == 0), R(0), R(1) / Rv(v))
    assert np.array_equal(take(n), d)
    xb = np.where(bnd, Rv(v), x1)
    assert np.array_equal(take(n), xb)
    r32 = np.where(bnd, np.float32(0), xb.astype(np.float32))
    assert np.array_equal(take(n), r32) and np.array_equal(take(n), np.zeros(n))
    assert np.array_equal(take(n), xb.astype(np.float64) + r32.astype(np.float64))
    assert np.array_equal(take(n), xb)
    assert o == out.size


def test_cg_vector_kernels_have_no_data_race(cg_exe_tsan, tmp_path):
    """The same sequence under ThreadSanitizer (block sums, the last block's
    completion of the CG update)."""
    _run_cg(cg_exe_tsan, tmp_path, 3000, "fp64", 4)
