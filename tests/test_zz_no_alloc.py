"""elm_advect_noalloc: the advection step for callers that cannot allocate
device memory at the call site (for example an application whose device
memory is handed out by its own pool, or a time-critical loop that cannot
take cudaMalloc's implicit synchronisation).  It runs the same kernels on the
same packed velocity records as elm_advect, so its output must equal the
regular path bit for bit, on two calls in a row, for 2D and 3D meshes, P2 and
P1 elements, and a mesh blended onto an annulus.  This file is collected last
on purpose."""
import ctypes

import pytest
import torch

from paper_2103_02388_gb300 import _lib, elm, inputs

pytestmark = pytest.mark.gpu

ANNULUS = (0.5, 1.5, 6, 0.0)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(mesh, u_old, u_new, T_old, T_new, dt, n_sub):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(lib.elm_advect_noalloc(mesh.handle, _ptr(u_old), _ptr(u_new), _ptr(T_old), _ptr(T_new),
                                      float(dt), int(n_sub), stream))


def _fields(mesh, dim):
    x = mesh.node_coords()
    dt_ = mesh.dtype
    if mesh.annulus is not None:
        u0 = 1.5 * (torch.tensor(x[:, ::-1].copy()) * torch.tensor([-1.0, 1.0]) + torch.tensor([0.3, -0.2]))
        u1 = u0 * 0.8 + torch.tensor([0.1, 0.2])
        T = torch.exp(-((torch.tensor(x) - torch.tensor([0.0, 1.0])) ** 2).sum(1) / 0.05)
        return u0.to(dt_).cuda(), u1.to(dt_).cuda(), T.to(dt_).cuda(), 0.05
    u0 = inputs.rotation_2d(x) if dim == 2 else inputs.cellular_flow(x)
    u1 = inputs.random_fourier(x, seed=4)
    T = inputs.gaussian(x, (0.35, 0.5, 0.5)[:dim], 0.15) if dim == 3 else inputs.slotted_cylinder(x)
    dt = inputs.dt_for_cfl(4.0, mesh.level, u1)
    return (torch.tensor(u0, dtype=dt_, device="cuda"), torch.tensor(u1, dtype=dt_, device="cuda"),
            torch.tensor(T, dtype=dt_, device="cuda"), dt)


CASES = [  # (dim, level, precision, order, annulus)
    (3, 3, "fp64", 2, None), (3, 3, "fp32", 2, None), (3, 4, "fp32", 1, None), (3, 4, "fp64", 1, None),
    (2, 5, "fp64", 2, None), (2, 5, "fp32", 2, None), (2, 6, "fp32", 1, None),
    (2, 3, "fp64", 2, ANNULUS), (2, 4, "fp64", 1, ANNULUS),
]


@pytest.mark.parametrize("dim,level,precision,order,annulus", CASES)
def test_noalloc_equals_advect(dim, level, precision, order, annulus):
    if annulus is not None:
        v, m = inputs.annulus_ring(6, 2)
    else:
        v, m = inputs.unit_cube() if dim == 3 else inputs.unit_square()
    mesh = elm.Mesh(v, m, level, precision, order=order, annulus=annulus)
    u0, u1, T, dt = _fields(mesh, dim)
    out = torch.full_like(T, float("nan"))
    # two calls in a row: steady, then time-dependent velocity
    for u_old, u_new, n_sub in ((u0, u0, 2), (u0, u1, 3)):
        mesh.set_velocity(u_old, u_new)
        ref = mesh.advect(T, dt, n_sub)
        _noalloc(mesh, u_old, u_new, T, out, dt, n_sub)
        torch.cuda.synchronize()
        mesh.status()
        assert torch.equal(out, ref)


def test_noalloc_rejects_meshes_beyond_the_limit():
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, 5, "fp32")          # 6 * (65*66*67/6) = 287,430 storage nodes: within
    u = torch.zeros((mesh.n_nodes, 3), dtype=torch.float32, device="cuda")
    T = torch.ones(mesh.n_nodes, dtype=torch.float32, device="cuda")
    out = torch.empty_like(T)
    _noalloc(mesh, u, u, T, out, 0.01, 1)
    torch.cuda.synchronize()
    assert torch.equal(out, T)
    big = elm.Mesh(v, m, 6, "fp32")           # 2,196,870 storage nodes: beyond 2^19
    ub = torch.zeros((big.n_nodes, 3), dtype=torch.float32, device="cuda")
    Tb = torch.ones(big.n_nodes, dtype=torch.float32, device="cuda")
    with pytest.raises(_lib.ElmError) as e:
        _noalloc(big, ub, ub, Tb, torch.empty_like(Tb), 0.01, 1)
    assert e.value.status == _lib.ELM_ERR_ARG
    assert b"static scratch limit" in _lib.load().elm_last_error()
