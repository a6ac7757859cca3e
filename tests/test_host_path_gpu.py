"""GPU tests of the host-buffer step (elm_advect_host): pinned host inputs and
result, copies pipelined on the mesh's own streams, the step launched in
pieces.  The result must equal the device step (elm_set_velocity +
elm_advect) bit for bit, since both run the same kernel on the same inputs,
and the oracle within the parity tolerance."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from _helpers import match_nodes, mesh_for, scalar_for, velocity_for
from paper_2103_02388_gb300 import _lib, elm, inputs

pytestmark = pytest.mark.gpu


def _fields(gm, vel="fourier", scal="gauss", seed=0):
    x = gm.node_coords()
    u = velocity_for(vel, x) if vel != "fourier" else inputs.random_fourier(x, seed=seed)
    T = scalar_for(scal, x)
    return (torch.tensor(u, dtype=gm.dtype).contiguous(), torch.tensor(T, dtype=gm.dtype).contiguous())


def _device_step(gm, T, u_old, dt, n_sub, u_new=None):
    uo = u_old.cuda()
    un = uo if u_new is None else u_new.cuda()
    gm.set_velocity(uo, un)
    out = gm.advect(T.cuda(), dt, n_sub)
    gm.status()
    return out.cpu()


def _single_triangle():
    return np.array([[0.0, 0.0], [1.0, 0.0], [0.3, 0.9]]), np.array([[0, 1, 2]])


@pytest.mark.parametrize("mesh,level,precision,order,steady", [
    ("cube", 3, "fp32", 2, True),
    ("cube", 3, "fp64", 2, False),
    ("cube", 4, "fp32", 1, True),
    ("square", 5, "fp64", 2, True),
    ("square_block", 3, "fp32", 1, False),
    ("cube_block", 2, "fp32", 2, True),
    ("triangle", 0, "fp64", 1, True),    # 2 work-list chunks: two of the four pieces are empty
    ("triangle", 0, "fp32", 2, False),
])
def test_host_step_equals_device_step(mesh, level, precision, order, steady):
    v, m = _single_triangle() if mesh == "triangle" else mesh_for(mesh)
    gm = elm.Mesh(v, m, level, precision, order=order, host_staging=True)
    u0, T = _fields(gm, seed=1)
    u1 = None if steady else _fields(gm, seed=2)[0]
    dt = inputs.dt_for_cfl(4.0, level, u0.double().numpy())
    n_sub = 2
    ref = _device_step(gm, T, u0, dt, n_sub, u1)
    pin = lambda t: None if t is None else t.pin_memory()
    out = gm.advect_host(pin(T), dt, n_sub, u_old=pin(u0), u_new=pin(u1))
    torch.cuda.synchronize()
    gm.status()
    assert torch.equal(out, ref)


def test_host_step_matches_oracle():
    v, m = mesh_for("cube")
    level = 3
    om = oracle.OracleMesh(v, m, level)
    gm = elm.Mesh(v, m, level, "fp64", host_staging=True)
    perm = match_nodes(om.coords, gm.unique_coords())
    u = velocity_for("cellular", om.coords)
    T = scalar_for("slotted", om.coords)
    dt = inputs.dt_for_cfl(4.0, level, u)
    umap = torch.tensor(gm.unique_map())

    def to_storage(a):
        g = np.empty_like(a)
        g[perm] = a
        return torch.tensor(g)[umap].contiguous().pin_memory()

    out = gm.advect_host(to_storage(T), dt, 2, u_old=to_storage(u))
    torch.cuda.synchronize()
    gm.status()
    owner = np.full(gm.n_unique, -1, np.int64)
    owner[gm.unique_map()[::-1]] = np.arange(gm.n_nodes)[::-1]
    got = out.numpy()[owner][perm]
    ref = om.advect(T, u, dt, 2)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(T).max()
    # every storage copy of a node holds the same value
    assert np.array_equal(out.numpy(), out.numpy()[owner][gm.unique_map()])


@pytest.mark.parametrize("form", ["feedback", "in_place", "ping_pong"])
def test_host_pipeline_of_steps(form):
    """Several calls enqueued without synchronising: each call's result is
    the next call's input, through the host."""
    v, m = mesh_for("cube")
    gm = elm.Mesh(v, m, 3, "fp32", host_staging=True)
    u, T = _fields(gm, seed=3)
    dt = inputs.dt_for_cfl(3.0, 3, u.double().numpy())
    steps = 6
    ref = T.clone()
    for _ in range(steps):
        ref = _device_step(gm, ref, u, dt, 1)
    u_h = u.pin_memory()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        if form == "feedback":
            cur = T.pin_memory()
            for _ in range(steps):
                cur = gm.advect_host(cur, dt, 1, u_old=u_h)
        elif form == "in_place":
            cur = T.pin_memory()
            for _ in range(steps):
                gm.advect_host(cur, dt, 1, u_old=u_h, out=cur)
        else:
            a, b = T.pin_memory(), torch.empty_like(T).pin_memory()
            for _ in range(steps):
                gm.advect_host(a, dt, 1, u_old=u_h, out=b)
                a, b = b, a
            cur = a
    stream.synchronize()
    gm.status()
    assert torch.equal(cur, ref)


def test_host_step_refuses_pageable_and_unstaged():
    v, m = mesh_for("square")
    gm = elm.Mesh(v, m, 2, "fp64", host_staging=True)
    u, T = _fields(gm)
    with pytest.raises(ValueError):
        gm.advect_host(T, 0.1, 1, u_old=u.pin_memory())          # pageable T
    lib = _lib.load()
    pinned = torch.empty(gm.n_nodes * 2, dtype=torch.float64).pin_memory()
    pageable = np.zeros(gm.n_nodes * 2)
    p = ctypes.c_void_p(pinned.data_ptr())
    q = pageable.ctypes.data_as(ctypes.c_void_p)
    assert lib.elm_advect_host(gm.handle, p, p, q, p, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert b"page-locked" in lib.elm_last_error()
    plain = elm.Mesh(v, m, 2, "fp64")
    assert lib.elm_advect_host(plain.handle, p, p, p, p, 0.1, 1, None) == _lib.ELM_ERR_STATE
    # a refused call leaves the mesh usable
    out = gm.advect_host(T.pin_memory(), 0.1, 1, u_old=u.pin_memory())
    torch.cuda.synchronize()
    assert torch.equal(out, _device_step(gm, T, u, 0.1, 1))


@pytest.mark.parametrize("precision,steady", [("fp32", True), ("fp64", False)])
def test_host_step_with_resident_velocity(precision, steady):
    """Both velocity pointers null: the mesh's current velocity stays on the
    device and only T moves.  A time loop of such calls equals the device
    loop bit for bit; a mesh with no velocity refuses the call."""
    v, m = mesh_for("cube")
    gm = elm.Mesh(v, m, 3, precision, host_staging=True)
    u0, T = _fields(gm, seed=3)
    u1 = None if steady else _fields(gm, seed=4)[0]
    dt = inputs.dt_for_cfl(4.0, 3, u0.double().numpy())
    bare = elm.Mesh(v, m, 3, precision, host_staging=True)
    with pytest.raises(_lib.ElmError) as e:
        bare.advect_host(T.pin_memory(), dt, 1)
    assert e.value.status == _lib.ELM_ERR_STATE
    # device loop
    gm.set_velocity(u0.cuda(), None if u1 is None else u1.cuda())
    ref = T.cuda()
    for _ in range(3):
        ref = gm.advect(ref, dt, 1)
    torch.cuda.synchronize()
    # host loop: the velocity given once, then T alone (in place)
    Th = T.clone().pin_memory()
    gm.advect_host(Th, dt, 1, u_old=u0.pin_memory(), u_new=None if u1 is None else u1.pin_memory(), out=Th)
    for _ in range(2):
        gm.advect_host(Th, dt, 1, out=Th)
    torch.cuda.synchronize()
    gm.status()
    assert torch.equal(Th, ref.cpu())
