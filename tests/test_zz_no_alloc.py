"""elm_advect_noalloc: the advection step for callers that cannot allocate
device memory at the call site (for example an application whose device
memory is handed out by its own pool, or a time-critical loop that cannot
take cudaMalloc's implicit synchronisation).  Its output must match the
regular elm_advect path on the same inputs, on two calls in a row.  This file
is collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_02388_gb300 import _lib, elm, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _noalloc(mesh, u_old, u_new, T_old, T_new, dt, n_sub):
    lib = _lib.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check(lib.elm_advect_noalloc(mesh.handle, _ptr(u_old), _ptr(u_new), _ptr(T_old), _ptr(T_new),
                                      float(dt), int(n_sub), stream))


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_noalloc_matches_advect(precision):
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, 3, precision)
    x = torch.tensor(mesh.node_coords())
    dt_ = mesh.dtype
    u0 = torch.tensor(inputs.cellular_flow(x.numpy()), dtype=dt_, device="cuda")
    u1 = torch.tensor(inputs.random_fourier(x.numpy(), seed=4), dtype=dt_, device="cuda")
    T = torch.tensor(inputs.slotted_sphere(x.numpy()), dtype=dt_, device="cuda")
    dt = inputs.dt_for_cfl(4.0, 3, u1.double().cpu().numpy())
    tol = TOL[precision] * float(T.abs().max())
    out = torch.empty_like(T)
    # two calls in a row, steady and then time-dependent velocity
    for u_old, u_new, n_sub in ((u0, u0, 2), (u0, u1, 3)):
        mesh.set_velocity(u_old, u_new)
        ref = mesh.advect(T, dt, n_sub)
        _noalloc(mesh, u_old, u_new, T, out, dt, n_sub)
        torch.cuda.synchronize()
        mesh.status()
        assert float((out - ref).abs().max()) <= tol


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
