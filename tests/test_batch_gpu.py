"""Batched form: one persistent launch (per element order) over many
independent P2 and P1 instances must give, for every instance, bitwise the
result of its own elm_advect call;
CUDA-graph replay of a batched time loop must equal the eager loop."""
import numpy as np
import pytest
import torch

from _helpers import mesh_for
from paper_2103_02388_gb300 import _lib, elm, inputs
from paper_2103_02388_gb300.autotune import tune_batch

pytestmark = pytest.mark.gpu


def _instances(precision):
    # (mesh, level, velocity, CFL, n_sub, element order): P2 and P1 instances mixed
    specs = [("square", 3, "rotation", 1.5, 1, 2), ("cube", 2, "fourier", 4.0, 2, 2), ("square", 5, "fourier", 8.0, 1, 2),
             ("cube", 3, "rotation", 0.5, 3, 2), ("cube_block", 1, "fourier", 6.0, 1, 2),
             ("square_block", 2, "rotation", 2.0, 2, 2), ("cube", 4, "fourier", 4.0, 1, 1),
             ("square", 6, "rotation", 3.0, 2, 1), ("cube_block", 2, "fourier", 5.0, 1, 1)]
    out = []
    for k, (mesh, level, vel, cfl, n_sub, order) in enumerate(specs):
        v, m = mesh_for(mesh)
        gm = elm.Mesh(v, m, level, precision, order=order)
        x = gm.node_coords()
        u = (inputs.rotation_2d(x) if x.shape[1] == 2 else inputs.rotation_3d(x)) if vel == "rotation" \
            else inputs.random_fourier(x, seed=10 + k)
        T = inputs.gaussian(x, (0.4, 0.5, 0.5)[:x.shape[1]], 0.15)
        ut = torch.tensor(u, dtype=gm.dtype, device="cuda")
        u2 = None
        if k % 3 == 1:  # some instances time-dependent
            u2 = torch.tensor(inputs.random_fourier(x, seed=50 + k), dtype=gm.dtype, device="cuda")
        gm.set_velocity(ut, u2)
        out.append((gm, torch.tensor(T, dtype=gm.dtype, device="cuda"),
                    inputs.dt_for_cfl(cfl, level, u), n_sub, (ut, u2)))
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_batch_equals_single_runs(precision):
    inst = _instances(precision)
    meshes = [i[0] for i in inst]
    T_old = [i[1] for i in inst]
    dts = [i[2] for i in inst]
    subs = [i[3] for i in inst]
    ref = [m.advect(T, dt, s) for m, T, dt, s in zip(meshes, T_old, dts, subs)]
    # launch shapes: resident blocks per SM (and with them the register
    # budget: 8 or more selects the 8-block kernel) and chunks per work item
    for bps, cpi in ((1, 1), (4, 2), (6, 4), (8, 1), (8, 3)):
        b = elm.Batch(meshes, bps, cpi)
        out = [torch.full_like(T, float("nan")) for T in T_old]
        b.advect(T_old, out, dts, subs)
        torch.cuda.synchronize()
        for m in meshes:
            m.status()
        for r, o in zip(ref, out):
            assert torch.equal(r, o)


def test_batch_graph_time_loop():
    inst = _instances("fp32")
    meshes = [i[0] for i in inst]
    dts = [i[2] for i in inst]
    subs = [i[3] for i in inst]
    a = [i[1].clone() for i in inst]
    c = [torch.empty_like(x) for x in a]
    b = elm.Batch(meshes, 4)
    steps = 6
    # eager reference
    ea, ec = [x.clone() for x in a], [torch.empty_like(x) for x in a]
    for _ in range(steps):
        b.advect(ea, ec, dts, subs)
        ea, ec = ec, ea
    torch.cuda.synchronize()
    # captured loop: ping-pong between a and c inside one graph
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        b.advect(a, c, dts, subs)  # warm-up outside the capture
    torch.cuda.current_stream().wait_stream(s)
    a = [i[1].clone() for i in inst]
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        x, y = a, c
        for _ in range(steps):
            b.advect(x, y, dts, subs)
            x, y = y, x
    a_init = [i[1] for i in inst]
    for dst, src in zip(a, a_init):
        dst.copy_(src)
    g.replay()
    torch.cuda.synchronize()
    final = a if steps % 2 == 0 else c
    for r, o in zip(ea, final):
        assert torch.equal(r, o)


def test_batch_errors():
    v, m = inputs.unit_cube()
    m64 = elm.Mesh(v, m, 1, "fp64")
    m32 = elm.Mesh(v, m, 1, "fp32")
    with pytest.raises(_lib.ElmError):
        elm.Batch([m64, m32])
    b = elm.Batch([m64])
    T = torch.ones(m64.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ElmError) as e:
        b.advect([T], [torch.empty_like(T)], [0.1], [1])
    assert e.value.status == _lib.ELM_ERR_STATE
    m64.set_velocity(torch.zeros((m64.n_nodes, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(_lib.ElmError):
        b.advect([T], [T], [0.1], [1])
    with pytest.raises(_lib.ElmError):
        b.advect([T], [torch.empty_like(T)], [0.1], [0])


def test_autotuner_picks_a_candidate(tmp_path):
    inst = _instances("fp32")
    meshes = [i[0] for i in inst]
    T_old = [i[1] for i in inst]
    out = [torch.empty_like(T) for T in T_old]
    res = tune_batch(meshes, T_old, out, [i[2] for i in inst], [i[3] for i in inst], blocks_per_sm=(1, 8),
                     chunks_per_item=(1, 3), reps=2, cache_path=str(tmp_path / "tune.json"))
    assert res["blocks_per_sm"] in (1, 8) and res["chunks_per_item"] in (1, 3)
    assert sorted(res["ms"]) == ["1:1", "1:3", "8:1", "8:3"]
    again = tune_batch(meshes, T_old, out, [i[2] for i in inst], [i[3] for i in inst], blocks_per_sm=(1, 8),
                       chunks_per_item=(1, 3), cache_path=str(tmp_path / "tune.json"))
    assert again == res
