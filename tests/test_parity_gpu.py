"""GPU parity: the CUDA advection step (through the C ABI) against the CPU
oracle, element by element on the same seeded inputs.

FP64: max |T_gpu - T_oracle| <= 1e-12 * max |T_old| per step.
FP32: max |T_gpu - T_oracle| <= 1e-5 * max |T_old| per step, where the
oracle (FP64) receives the FP32-rounded inputs the GPU computes on.
"""
import numpy as np
import pytest
import torch

import oracle
from _helpers import match_nodes, mesh_for, scalar_for, velocity_for
from paper_2103_02388_gb300 import _lib, elm, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


class Pair:
    """The same mesh on both sides, with the node permutation between them."""

    def __init__(self, mesh, level, precision="fp64", order=2):
        v, m = mesh_for(mesh) if isinstance(mesh, str) else mesh
        self.om = oracle.OracleMesh(v, m, level, order=order)
        self.gm = elm.Mesh(v, m, level, precision, order=order)
        self.perm = match_nodes(self.om.coords, self.gm.unique_coords())
        self.precision = precision
        self.level = level
        self.x = self.om.coords

    def rounded(self, a):
        return a.astype(np.float32).astype(np.float64) if self.precision == "fp32" else a

    def to_gpu(self, a):
        g = np.empty_like(a)
        g[self.perm] = a
        t = torch.tensor(g, dtype=self.gm.dtype, device="cuda")
        return self.gm.to_storage(t)

    def from_gpu(self, t):
        return self.gm.to_unique(t).double().cpu().numpy()[self.perm]

    def step(self, T, u, dt, n_sub=1, u_new=None, check_copies=True):
        """One step on both sides; returns (gpu, oracle) in oracle node order."""
        T, u = self.rounded(T), self.rounded(u)
        u_new = None if u_new is None else self.rounded(u_new)
        us = self.to_gpu(u)
        un = us if u_new is None else self.to_gpu(u_new)
        self.gm.set_velocity(us, un)
        out = self.gm.advect(self.to_gpu(T), dt, n_sub)
        self.gm.status()
        if check_copies:
            umap = torch.tensor(self.gm.unique_map(), device="cuda")
            uniq = self.gm.to_unique(out)
            assert torch.equal(uniq[umap], out), "storage copies of a node disagree"
        ref = self.om.advect(T, u, dt, n_sub, u_new=u_new)
        return self.from_gpu(out), ref


def _err(got, ref, T):
    return np.abs(got - ref).max() / max(np.abs(T).max(), 1e-300)


@pytest.mark.parametrize("mesh,level,vel,scal,cfl,n_sub", [
    ("square", 5, "rotation", "gauss", None, 1),      # circular advection, dt = 1/200
    ("square", 3, "rotation", "quadratic", 3.0, 3),
    ("square_block", 3, "fourier", "gauss", 6.0, 2),
    ("cube", 3, "cellular", "slotted", 1.0, 1),
    ("cube", 3, "cellular", "slotted", 4.0, 2),
    ("cube", 3, "cellular", "slotted", 8.0, 4),
    ("cube", 4, "fourier", "gauss", 4.0, 1),
    ("cube", 2, "rotation", "gauss", 5.0, 2),           # leaves the cube: clamping
    ("cube_block", 2, "fourier", "gauss", 8.0, 2),      # 48 perturbed macros: walk
    ("cube_block", 1, "rotation", "slotted", 3.0, 1),
])
def test_fp64_parity(mesh, level, vel, scal, cfl, n_sub):
    P = Pair(mesh, level, "fp64")
    u = velocity_for(vel, P.x)
    T = scalar_for(scal, P.x)
    dt = 1 / 200 if cfl is None else inputs.dt_for_cfl(cfl, level, u)
    got, ref = P.step(T, u, dt, n_sub)
    assert _err(got, ref, T) <= TOL["fp64"]


@pytest.mark.parametrize("mesh,level,vel,scal,cfl,n_sub", [
    ("square", 5, "rotation", "gauss", None, 1),
    ("square", 6, "fourier", "gauss", 4.0, 2),
    ("cube", 4, "fourier", "gauss", 4.0, 1),
    ("cube", 4, "cellular", "slotted", 8.0, 2),
    ("cube_block", 2, "fourier", "gauss", 8.0, 1),
])
def test_fp32_parity(mesh, level, vel, scal, cfl, n_sub):
    P = Pair(mesh, level, "fp32")
    u = velocity_for(vel, P.x)
    T = scalar_for(scal, P.x)
    dt = 1 / 200 if cfl is None else inputs.dt_for_cfl(cfl, level, u)
    got, ref = P.step(T, u, dt, n_sub)
    assert _err(got, ref, T) <= TOL["fp32"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_time_dependent_velocity(precision):
    P = Pair("cube", 3, precision)
    u0 = inputs.cellular_flow(P.x)
    u1 = inputs.random_fourier(P.x, seed=4)
    T = scalar_for("gauss", P.x)
    dt = inputs.dt_for_cfl(3.0, 3, u1)
    got, ref = P.step(T, u0, dt, 3, u_new=u1)
    assert _err(got, ref, T) <= TOL[precision]


@pytest.mark.parametrize("mesh,level", [("square", 0), ("square", 1), ("cube", 0), ("cube", 1)])
def test_smallest_levels(mesh, level):
    P = Pair(mesh, level, "fp64")
    u = velocity_for("fourier", P.x)
    T = scalar_for("quadratic", P.x)
    got, ref = P.step(T, u, 0.3, 2)
    assert _err(got, ref, T) <= TOL["fp64"]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_zero_dt_and_zero_velocity_are_identity(precision):
    P = Pair("cube", 2, precision)
    T = P.rounded(scalar_for("quadratic", P.x))
    u = velocity_for("fourier", P.x)
    got, _ = P.step(T, u, 0.0, 1)
    tol = 8 * np.finfo(np.float64 if precision == "fp64" else np.float32).eps
    assert np.abs(got - T).max() <= tol * np.abs(T).max()
    got, _ = P.step(T, np.zeros_like(P.x), 0.5, 2)
    assert np.abs(got - T).max() <= tol * np.abs(T).max()


def test_accumulated_revolution_fp64():
    """Config of the circular-advection benchmark: 2D level 5, 200 steps of
    dt = 1/200 (one revolution), both sides run independently."""
    P = Pair("square", 5, "fp64")
    u = inputs.rotation_2d(P.x)
    T0 = inputs.gaussian(P.x, (0.25, 0.5), 0.05)
    us = P.to_gpu(u)
    P.gm.set_velocity(us)
    Tg = P.to_gpu(T0)
    To = T0.copy()
    worst = 0.0
    for _ in range(200):
        Tg = P.gm.advect(Tg, 1 / 200)
        To = P.om.advect(To, u, 1 / 200)
        worst = max(worst, np.abs(P.from_gpu(Tg) - To).max())
    P.gm.status()
    assert worst <= 1e-11
    # and the scheme itself: H0 error after one revolution is small
    assert P.om.metrics(To, T0, T0)["h0"] < 0.03


def test_largest_2d_level_interfaces():
    """2D level 9: lattice coordinates reach 1024, the widest owner record.
    Storage copies agree and sampled nodes (all of the diagonal interface,
    both corners on it) match the oracle."""
    P = Pair("square", 9)
    u = inputs.rotation_2d(P.x, omega=1.0) + 0.1
    T = inputs.hill(P.x)
    dt = inputs.dt_for_cfl(3.0, 9, u)
    P.gm.set_velocity(P.to_gpu(u))
    out = P.gm.advect(P.to_gpu(T), dt, 1)
    P.gm.status()
    umap = torch.tensor(P.gm.unique_map(), device="cuda")
    assert torch.equal(P.gm.to_unique(out)[umap], out), "storage copies of a node disagree"
    got = P.from_gpu(out)
    diag = np.flatnonzero(np.abs(P.x[:, 0] - P.x[:, 1]) < 1e-12)
    idx = np.union1d(diag, np.random.default_rng(0).choice(P.om.n_nodes, 2000, replace=False))
    ref = P.om.advect_nodes(T, u, dt, idx, 1)
    assert np.abs(got[idx] - ref).max() <= TOL["fp64"] * np.abs(T).max()


@pytest.mark.parametrize("precision,steps", [("fp64", 62), ("fp64", 628), ("fp32", 628)])
def test_lookback_infinity(precision, steps):
    """Look-back b = infinity (Sec. 2.3.3, Table 2): one revolution of the hill
    traced back to c0 in a single call with one RK4 substep per time step.
    FP64 within 1e-12 of the oracle.  FP32: each of the 4 * steps stage
    updates of the offset (|d| <= 0.75) rounds by at most 2^-24 |d|, so the
    departure point moves by at most 4 * 628 * 0.75 * 2^-24 ~ 1.1e-4 and T by
    that times max |grad c0| = pi / (4 * 0.15) ~ 5.2: 6e-4 (linear worst
    case, the oracle getting the FP32-rounded inputs)."""
    P = Pair("square", 6, precision)
    u = P.rounded(inputs.rotation_2d(P.x, omega=1.0))
    c0 = P.rounded(inputs.hill(P.x))
    P.gm.set_velocity(P.to_gpu(u))
    out = P.gm.advect_lookback(P.to_gpu(c0), 2 * np.pi / steps, steps)
    P.gm.status()
    got = P.from_gpu(out)
    ref = P.om.advect(c0, u, 2 * np.pi, n_sub=steps)
    tol = TOL["fp64"] if precision == "fp64" else 6e-4
    assert _err(got, ref, c0) <= tol
    if precision == "fp64":
        # the paper's error after one revolution (Table 2, b = infinity)
        paper = {62: 9.62e-7, 628: 9.13e-11}[steps]
        assert abs(P.om.metrics(got, c0, c0)["h0"] / paper - 1.0) < 0.02


def test_lookback_needs_steady_velocity():
    P = Pair("square", 2)
    u = inputs.rotation_2d(P.x, omega=1.0)
    P.gm.set_velocity(P.to_gpu(u), P.to_gpu(0.5 * u))
    with pytest.raises(ValueError):
        P.gm.advect_lookback(P.to_gpu(inputs.hill(P.x)), 0.1, 4)


@pytest.mark.parametrize("precision,level,n_sub,cfl,order", [("fp64", 6, 2, 4.0, 2), ("fp32", 7, 1, 4.0, 2),
                                                              ("fp32", 8, 1, 4.0, 1)])
def test_full_size_sampled(precision, level, n_sub, cfl, order):
    """The benchmark sizes (3D level 6 FP64, level 7 FP32, and P1 at its
    largest level 8, 257^3 nodes), checked on 3000 sampled nodes the oracle
    evaluates one by one."""
    P = Pair("cube", level, precision, order=order)
    if precision == "fp64":
        u = inputs.cellular_flow(P.x)
        T = inputs.slotted_sphere(P.x)
    else:
        u = inputs.random_fourier(P.x, seed=3)
        T = inputs.gaussian(P.x, (0.35, 0.5, 0.5), 0.1)
    u, T = P.rounded(u), P.rounded(T)
    dt = inputs.dt_for_cfl(cfl, level, u)
    us = P.to_gpu(u)
    P.gm.set_velocity(us)
    out = P.gm.advect(P.to_gpu(T), dt, n_sub)
    P.gm.status()
    got = P.from_gpu(out)
    rng = np.random.default_rng(0)
    idx = rng.choice(P.om.n_nodes, 3000, replace=False)
    ref = P.om.advect_nodes(T, u, dt, idx, n_sub)
    assert np.abs(got[idx] - ref).max() <= TOL[precision] * np.abs(T).max()


# ---------------------------------------------------------------------------
# Error behaviour (no GPU fault is provoked: conditions are flags and codes).
# ---------------------------------------------------------------------------


def test_nonfinite_velocity_is_reported():
    v, m = inputs.unit_cube()
    gm = elm.Mesh(v, m, 2, "fp64")
    u = torch.zeros((gm.n_nodes, 3), dtype=torch.float64, device="cuda")
    u[17, 1] = float("nan")
    gm.set_velocity(u)
    T = torch.ones(gm.n_nodes, dtype=torch.float64, device="cuda")
    gm.advect(T, 0.1, 1)
    with pytest.raises(_lib.ElmError) as e:
        gm.status()
    assert e.value.status == _lib.ELM_ERR_NONFINITE
    gm.status()  # flags were cleared


def test_walk_limit_is_reported_not_hung():
    """A step that crosses more macros than the walk limit allows returns a
    flag instead of looping."""
    v, m = inputs.square_block(48)
    gm = elm.Mesh(v, m, 0, "fp64")
    u = torch.zeros((gm.n_nodes, 2), dtype=torch.float64, device="cuda")
    u[:, 0] = 1.0
    u[:, 1] = 0.3
    gm.set_velocity(u)
    T = torch.ones(gm.n_nodes, dtype=torch.float64, device="cuda")
    gm.advect(T, 0.9, 1)
    with pytest.raises(_lib.ElmError) as e:
        gm.status()
    assert e.value.status == _lib.ELM_ERR_WALK_LIMIT


def test_argument_errors():
    v, m = inputs.unit_square()
    gm = elm.Mesh(v, m, 2, "fp64")
    T = torch.ones(gm.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ElmError) as e:
        gm.advect(T, 0.1)
    assert e.value.status == _lib.ELM_ERR_STATE          # no velocity yet
    gm.set_velocity(torch.zeros((gm.n_nodes, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(_lib.ElmError) as e:
        gm.advect(T, 0.1, out=T)
    assert e.value.status == _lib.ELM_ERR_ARG            # aliasing
    with pytest.raises(_lib.ElmError):
        gm.advect(T, 0.1, n_sub=0)
    with pytest.raises(_lib.ElmError):
        gm.advect(T, float("nan"))
    with pytest.raises(_lib.ElmError):
        gm.advect(T, -1.0)
    with pytest.raises(_lib.ElmError):
        gm.advect(T, 0.1, n_sub=65537)                   # above ELM_MAX_SUBSTEPS


# ---------------------------------------------------------------------------
# Linear (P1) elements (Sec. 3.1) and look-back over a time-dependent
# velocity (Sec. 2.3.3) through elm_trace / elm_trace_eval.
# ---------------------------------------------------------------------------


@pytest.mark.parametrize("mesh,level,vel,scal,cfl,n_sub,precision", [
    ("square", 6, "rotation", "gauss", 3.0, 1, "fp64"),
    ("square_block", 4, "fourier", "slotted", 6.0, 2, "fp64"),
    ("cube", 4, "cellular", "slotted", 4.0, 2, "fp64"),
    ("cube", 5, "fourier", "gauss", 8.0, 1, "fp64"),
    ("cube_block", 2, "fourier", "gauss", 8.0, 2, "fp64"),
    ("cube", 2, "rotation", "gauss", 5.0, 2, "fp64"),     # leaves the cube: clamping
    ("square", 7, "fourier", "gauss", 4.0, 2, "fp32"),
    ("cube", 5, "fourier", "gauss", 4.0, 1, "fp32"),
    ("cube_block", 2, "cellular", "slotted", 8.0, 1, "fp32"),
])
def test_p1_parity(mesh, level, vel, scal, cfl, n_sub, precision):
    P = Pair(mesh, level, precision, order=1)
    u = velocity_for(vel, P.x)
    T = scalar_for(scal, P.x)
    dt = inputs.dt_for_cfl(cfl, level, u)
    got, ref = P.step(T, u, dt, n_sub)
    assert _err(got, ref, T) <= TOL[precision]


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_p1_time_dependent_velocity(precision):
    P = Pair("cube", 4, precision, order=1)
    u0 = inputs.cellular_flow(P.x)
    u1 = inputs.random_fourier(P.x, seed=4)
    T = scalar_for("gauss", P.x)
    got, ref = P.step(T, u0, inputs.dt_for_cfl(3.0, 4, u1), 3, u_new=u1)
    assert _err(got, ref, T) <= TOL[precision]


def test_p1_table1_lookback_infinity():
    """Table 1, 'MMOC P1 (b = infinity)': three bodies, one revolution in one
    trace of 6283 RK4 substeps on 129 x 129 P1 nodes; the printed H0 is at
    round-off level (1.38e-13), and the GPU matches the oracle to 1e-12."""
    P = Pair("square", 7, "fp64", order=1)
    u = inputs.rotation_2d(P.x, omega=1.0)
    c0 = inputs.three_bodies(P.x)
    P.gm.set_velocity(P.to_gpu(u))
    got = P.from_gpu(P.gm.advect_lookback(P.to_gpu(c0), 2 * np.pi / 6283, 6283))
    P.gm.status()
    assert P.om.metrics(got, c0, c0)["h0"] < 3 * 1.38e-13
    ref = P.om.advect(c0, u, 2 * np.pi, n_sub=6283)
    assert _err(got, ref, c0) <= TOL["fp64"]


def _trace_both(P, c0, fields, tau, n_sub=1):
    """b = infinity over len(fields) - 1 intervals (newest first) on both
    sides; returns (T_gpu, T_oracle, D_gpu, X_oracle) in oracle node order."""
    us = [P.to_gpu(P.rounded(f)) for f in fields]
    D = None
    bufs = [torch.empty((P.gm.n_nodes, P.gm.dim), dtype=P.gm.dtype, device="cuda") for _ in range(2)]
    for j, k in enumerate(range(len(fields) - 1, 0, -1)):
        P.gm.set_velocity(us[k - 1], us[k])
        D = P.gm.trace(D, tau, n_sub, out=bufs[j % 2])
    Tg = P.gm.trace_eval(D, P.to_gpu(P.rounded(c0)))
    P.gm.status()
    X = P.x.copy()
    for k in range(len(fields) - 1, 0, -1):
        X = P.om.trace(X, P.rounded(fields[k - 1]), tau, n_sub, u_new=P.rounded(fields[k]))
    To = P.om.eval(P.rounded(c0), X)
    Dg = P.gm.to_unique(D).double().cpu().numpy()[P.perm]
    return P.from_gpu(Tg), To, Dg, X


@pytest.mark.parametrize("order,level,precision", [(1, 4, "fp64"), (2, 3, "fp64"), (1, 4, "fp32"), (2, 3, "fp32")])
def test_trace_swirl_parity(order, level, precision):
    """The swirling flow of Sec. 3.3 (time-dependent), b = infinity over 10
    intervals of tau = 0.15: departure offsets and the final field against
    the oracle's trace continuation."""
    P = Pair("cube", level, precision, order=order)
    c0 = inputs.gaussian(P.x, (0.35, 0.5, 0.5), 0.1)
    tau = 0.15
    fields = [inputs.swirl_3d(P.x, k * tau) for k in range(11)]
    Tg, To, Dg, X = _trace_both(P, c0, fields, tau, n_sub=2)
    dtol = 1e-12 if precision == "fp64" else 2e-5
    assert np.abs((P.x + Dg) - X).max() <= dtol
    assert _err(Tg, To, c0) <= (TOL["fp64"] if precision == "fp64" else 2e-4)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_trace_then_eval_equals_advect(precision):
    """One interval traced from the nodes and evaluated is the step itself,
    bit for bit (same arithmetic, the offsets stored in the mesh precision)."""
    v, m = inputs.cube_block(2, perturb=0.25, seed=7)
    gm = elm.Mesh(v, m, 2, precision)
    x = gm.node_coords()
    u0 = torch.tensor(inputs.cellular_flow(x), dtype=gm.dtype, device="cuda")
    u1 = torch.tensor(inputs.random_fourier(x, seed=2), dtype=gm.dtype, device="cuda")
    T = torch.tensor(inputs.gaussian(x, (0.35, 0.5, 0.5), 0.1), dtype=gm.dtype, device="cuda")
    for pair in ((u0, u0), (u0, u1)):
        gm.set_velocity(*pair)
        ref = gm.advect(T, 0.07, 2)
        got = gm.trace_eval(gm.trace(None, 0.07, 2), T)
        gm.status()
        assert torch.equal(got, ref)


def test_trace_copies_agree_and_errors():
    P = Pair("cube_block", 1, "fp64", order=1)
    u = P.to_gpu(inputs.random_fourier(P.x, seed=5))
    P.gm.set_velocity(u)
    D1 = P.gm.trace(None, 0.2, 1)
    D2 = P.gm.trace(D1, 0.2, 1)
    umap = torch.tensor(P.gm.unique_map(), device="cuda")
    assert torch.equal(P.gm.to_unique(D2)[umap], D2)
    with pytest.raises(_lib.ElmError):
        P.gm.trace(D1, 0.2, 1, out=D1)             # in place: D_in and D_out overlap
    with pytest.raises(_lib.ElmError):
        P.gm.trace(D1, float("nan"), 1)
    with pytest.raises(_lib.ElmError):
        P.gm.trace(D1, 0.2, 0)
    T = P.to_gpu(inputs.random_linear(P.x, seed=1))
    with pytest.raises(_lib.ElmError):
        P.gm.trace_eval(D1, T, out=T)              # T_src and T_dst overlap


def test_table3_swirl_gpu():
    """Table 3 (swirling flow, P1, b = infinity) on the GPU: the 33^3 rows
    against the oracle (FP64, 1e-12) and all six rows against the printed
    magnitudes (H0 within a factor 3, var = 1), including the 129^3 rows
    (2,146,689 nodes)."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "table3_swirl_p1_binf.json")) as f:
        rows = json.load(f)["rows"]
    for level in (5, 7):
        P = Pair("cube", level, "fp64", order=1)
        assert P.gm.n_unique == {5: 35937, 7: 2146689}[level]
        c0 = inputs.half_space(P.x)
        c0g = P.to_gpu(c0)
        for ref in [r for r in rows if r["dofs"] == P.gm.n_unique]:
            tau = ref["tau"]
            K = int(round(1.5 / tau))
            fields = [P.to_gpu(inputs.swirl_3d(P.x, k * tau)) for k in range(K + 1)]
            got = P.from_gpu(P.gm.advect_lookback_unsteady(c0g, fields, tau))
            P.gm.status()
            r = P.om.metrics(got, c0, c0)
            assert ref["h0"] / 3 < r["h0"] < 3 * ref["h0"]
            assert abs(r["var"] - 1.0) < 1e-12
            if level == 5:
                X = P.x.copy()
                for k in range(K, 0, -1):
                    X = P.om.trace(X, inputs.swirl_3d(P.x, (k - 1) * tau), tau, 1,
                                   u_new=inputs.swirl_3d(P.x, k * tau))
                assert _err(got, P.om.eval(c0, X), c0) <= TOL["fp64"]


@pytest.mark.parametrize("precision,order", [("fp64", 2), ("fp32", 1)])
def test_shift_velocity_equals_set_velocity(precision, order):
    """elm_shift_velocity (the next older look-back interval: the current
    u_old becomes u_new, a new u_old is packed) traces exactly as
    elm_set_velocity with that pair, after a time-dependent pair and after a
    steady field."""
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, 3, precision, order=order)
    x = mesh.node_coords()
    f = [torch.tensor(inputs.swirl_3d(x, t), dtype=mesh.dtype, device="cuda") for t in (0.0, 0.1, 0.2)]
    tau = 0.1
    mesh.set_velocity(f[1], f[2])
    D1 = mesh.trace(None, tau, 2)
    mesh.shift_velocity(f[0])                       # (f0, f1)
    got = mesh.trace(D1, tau, 2)
    mesh.set_velocity(f[0], f[1])
    ref = mesh.trace(D1, tau, 2)
    assert torch.equal(got, ref)
    mesh.set_velocity(f[2])                         # steady f2, then (f1, f2)
    mesh.shift_velocity(f[1])
    got = mesh.trace(None, tau, 2)
    mesh.set_velocity(f[1], f[2])
    assert torch.equal(got, mesh.trace(None, tau, 2))
    mesh.status()
