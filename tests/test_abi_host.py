"""CPU tests of the C ABI: the library loads and exports every declared entry
point, and the host-side mesh logic (storage layout, unique numbering,
ownership, topology checks, argument errors) is right.  No GPU needed."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2103_02388_gb300 import _lib, inputs
from paper_2103_02388_gb300.build import build_library

import oracle
from _helpers import match_nodes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_library()
    return _lib.load()


def _declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names |= set(re.findall(r"\b(elm_\w+)\s*\(", text))
    return names


def test_every_declared_symbol_is_exported(lib):
    declared = _declared_functions()
    assert {"elm_mesh_create", "elm_advect", "elm_set_velocity", "elm_get_status"} <= declared
    for name in declared:
        assert hasattr(lib, name), name
    # the binding covers every declared entry point
    assert declared == {n for n, _, _ in _lib.SIGNATURES}


def _host_mesh(lib, v, m, level, precision=_lib.ELM_FP64):
    v = np.ascontiguousarray(v, np.float64)
    m = np.ascontiguousarray(m, np.int64)
    h = ctypes.c_void_p()
    st = lib.elm_mesh_create(v.shape[1], v.shape[0], v.ctypes.data_as(ctypes.c_void_p), m.shape[0],
                             m.ctypes.data_as(ctypes.c_void_p), level, precision | _lib.ELM_HOST_ONLY,
                             ctypes.byref(h))
    return st, h


@pytest.mark.parametrize("mesh,level", [("square", 0), ("square", 4), ("cube", 0), ("cube", 3),
                                        ("block", 2), ("sqblock", 3)])
def test_host_mesh_matches_oracle_nodes(lib, mesh, level):
    from paper_2103_02388_gb300 import elm
    v, m = {"square": inputs.unit_square, "cube": inputs.unit_cube,
            "block": lambda: inputs.cube_block(2, 0.3, 1),
            "sqblock": lambda: inputs.square_block(3, 0.3, 1)}[mesh]()
    gm = elm.Mesh(v, m, level, host_only=True)
    om = oracle.OracleMesh(v, m, level)
    assert gm.n_unique == om.n_nodes
    d = v.shape[1]
    M = 2 ** (level + 1)
    npm = (M + 1) * (M + 2) * (M + 3) // 6 if d == 3 else (M + 1) * (M + 2) // 2
    assert gm.n_nodes == m.shape[0] * npm
    perm = match_nodes(om.coords, gm.unique_coords())
    assert sorted(perm) == list(range(gm.n_unique))
    # every storage copy of a node sits at that node's coordinates
    umap = gm.unique_map()
    coords = gm.node_coords()
    ucoords = gm.unique_coords()
    assert np.abs(coords - ucoords[umap]).max() < 1e-12
    # owners are the first storage occurrence (lowest macro)
    first = np.full(gm.n_unique, -1)
    for s in range(gm.n_nodes - 1, -1, -1):
        first[umap[s]] = s
    assert np.all(np.diff(first) > 0)


def test_storage_layout_is_packed_rows(lib):
    from paper_2103_02388_gb300 import elm
    v, m = inputs.unit_cube()
    gm = elm.Mesh(v, m, 1, host_only=True)
    coords = gm.node_coords()
    M = 4
    P = v[np.sort(m[0])]
    k = 0
    for p1 in range(M + 1):
        for p2 in range(p1 + 1):
            for p3 in range(p2 + 1):
                s = np.array([p1, p2, p3]) / M
                x = P[0] + s[0] * (P[1] - P[0]) + s[1] * (P[2] - P[1]) + s[2] * (P[3] - P[2])
                assert np.allclose(coords[k], x, atol=1e-15)
                k += 1


def test_topology_and_argument_errors(lib):
    v, m = inputs.unit_cube()
    st, h = _host_mesh(lib, v, m, 8)
    assert st == _lib.ELM_ERR_ARG                       # level out of range in 3D
    st, h = _host_mesh(lib, v, m, -1)
    assert st == _lib.ELM_ERR_ARG
    bad = m.copy()
    bad[0, 1] = bad[0, 0]
    st, h = _host_mesh(lib, v, bad, 1)
    assert st == _lib.ELM_ERR_TOPOLOGY                  # repeated vertex
    flat = v.copy()
    flat[:, 2] = 0.0
    st, h = _host_mesh(lib, flat, m, 1)
    assert st == _lib.ELM_ERR_TOPOLOGY                  # degenerate macros
    triple = np.vstack([m, m[:1]])
    st, h = _host_mesh(lib, v, triple, 1)
    assert st == _lib.ELM_ERR_TOPOLOGY                  # face shared by 3 macros
    oob = m.copy()
    oob[2, 3] = 99
    st, h = _host_mesh(lib, v, oob, 1)
    assert st == _lib.ELM_ERR_ARG
    nan = v.copy()
    nan[3, 0] = np.nan
    st, h = _host_mesh(lib, nan, m, 1)
    assert st == _lib.ELM_ERR_ARG
    st, h = _host_mesh(lib, v, m, 1, precision=7)
    assert st == _lib.ELM_ERR_ARG
    assert b"precision" in lib.elm_last_error()


@pytest.mark.parametrize("mesh,level", [("square", 0), ("square", 5), ("cube", 1), ("cube", 3), ("block", 2)])
def test_p1_host_mesh_matches_oracle_nodes(lib, mesh, level):
    """ELM_P1: nodes are the micro vertices, M = 2^L lattice points per edge."""
    from paper_2103_02388_gb300 import elm
    v, m = {"square": inputs.unit_square, "cube": inputs.unit_cube,
            "block": lambda: inputs.cube_block(2, 0.3, 1)}[mesh]()
    gm = elm.Mesh(v, m, level, host_only=True, order=1)
    om = oracle.OracleMesh(v, m, level, order=1)
    assert gm.n_unique == om.n_nodes
    M = 2 ** level
    d = v.shape[1]
    npm = (M + 1) * (M + 2) * (M + 3) // 6 if d == 3 else (M + 1) * (M + 2) // 2
    assert gm.n_nodes == m.shape[0] * npm
    perm = match_nodes(om.coords, gm.unique_coords())
    assert sorted(perm) == list(range(gm.n_unique))
    assert np.abs(gm.node_coords() - gm.unique_coords()[gm.unique_map()]).max() < 1e-12


def test_p1_argument_errors(lib):
    v, m = inputs.unit_cube()
    st, h = _host_mesh(lib, v, m, 8, precision=_lib.ELM_FP64 | _lib.ELM_P1)
    assert st == _lib.ELM_OK                            # P1 goes one level finer
    lib.elm_mesh_destroy(h)
    st, h = _host_mesh(lib, v, m, 9, precision=_lib.ELM_FP64 | _lib.ELM_P1)
    assert st == _lib.ELM_ERR_ARG
    st, h = _host_mesh(lib, v, m, 2, precision=_lib.ELM_FP32 | _lib.ELM_P1 | _lib.ELM_ADJOINT)
    assert st == _lib.ELM_OK                            # the adjoint covers P1 too
    lib.elm_mesh_destroy(h)


def test_host_only_mesh_refuses_device_calls(lib):
    v, m = inputs.unit_square()
    st, h = _host_mesh(lib, v, m, 2)
    assert st == _lib.ELM_OK
    fake = ctypes.c_void_p(16)
    assert lib.elm_set_velocity(h, fake, fake, None) == _lib.ELM_ERR_STATE
    assert lib.elm_advect(h, fake, ctypes.c_void_p(4096), 0.1, 1, None) == _lib.ELM_ERR_STATE
    assert lib.elm_get_status(h, None) == _lib.ELM_ERR_STATE
    assert lib.elm_trace(h, None, ctypes.c_void_p(4096), 0.1, 1, None) == _lib.ELM_ERR_STATE
    assert lib.elm_trace_eval(h, fake, fake, ctypes.c_void_p(1 << 20), None) == _lib.ELM_ERR_STATE
    assert lib.elm_trace(h, None, None, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect(None, fake, fake, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_mesh_destroy(h) == _lib.ELM_OK
    assert lib.elm_mesh_num_nodes(None) == 0


def test_host_buffer_step_argument_errors(lib):
    v, m = inputs.unit_cube()
    st, h = _host_mesh(lib, v, m, 2, precision=_lib.ELM_FP32 | _lib.ELM_HOST_STAGING)
    assert st == _lib.ELM_OK                            # a host-only mesh sets up no staging
    fake = ctypes.c_void_p(4096)
    assert lib.elm_advect_host(h, fake, fake, fake, fake, 0.1, 1, None) == _lib.ELM_ERR_STATE
    assert b"host-only" in lib.elm_last_error()
    assert lib.elm_advect_host(h, None, fake, fake, fake, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect_host(h, fake, fake, fake, None, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect_host(h, fake, fake, fake, fake, float("nan"), 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect_host(h, fake, fake, fake, fake, -1.0, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect_host(h, fake, fake, fake, fake, 0.1, 0, None) == _lib.ELM_ERR_ARG
    assert lib.elm_advect_host(None, fake, fake, fake, fake, 0.1, 1, None) == _lib.ELM_ERR_ARG
    assert lib.elm_mesh_destroy(h) == _lib.ELM_OK


def test_missing_library_fails_loudly(tmp_path):
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(ImportError):
            _lib.load(str(tmp_path / "libelm.so"))
    finally:
        _lib._lib = saved


@pytest.mark.parametrize("order", [2, 1])
def test_blended_annulus_host_coordinates(lib, order):
    """elm_mesh_set_annulus: node coordinates become physical and equal the
    oracle's blended nodes (matched as point sets)."""
    from paper_2103_02388_gb300 import elm
    v, m = inputs.annulus_ring(6, 2)
    gm = elm.Mesh(v, m, 3, host_only=True, order=order, annulus=(0.5, 1.5, 6, 0.0))
    om = oracle.OracleMesh(v, m, 3, order=order, annulus=(0.5, 1.5, 6, 0.0))
    perm = match_nodes(om.coords, gm.unique_coords(), tol=1e-12)
    assert sorted(perm) == list(range(gm.n_unique))
    r = np.hypot(*gm.node_coords().T)
    assert abs(r.min() - 0.5) < 1e-14 and abs(r.max() - 1.5) < 1e-14


def test_blended_annulus_argument_errors(lib):
    v, m = inputs.annulus_ring(6, 2)
    st, h = _host_mesh(lib, v, m, 2)
    assert lib.elm_mesh_set_annulus(h, 0.5, 1.5, 5, 0.0) == _lib.ELM_ERR_TOPOLOGY   # wrong sector count
    assert lib.elm_mesh_set_annulus(h, 0.6, 1.5, 6, 0.0) == _lib.ELM_ERR_TOPOLOGY   # radius outside
    assert lib.elm_mesh_set_annulus(h, 1.5, 0.5, 6, 0.0) == _lib.ELM_ERR_ARG
    assert lib.elm_mesh_set_annulus(h, 0.5, 1.5, 6, 0.0) == _lib.ELM_OK
    assert lib.elm_mesh_set_annulus(h, 0.5, 1.5, 6, 0.0) == _lib.ELM_ERR_STATE      # twice
    st, h32 = _host_mesh(lib, v, m, 2, precision=_lib.ELM_FP32)
    assert lib.elm_mesh_set_annulus(h32, 0.5, 1.5, 6, 0.0) == _lib.ELM_ERR_ARG     # FP64 only
    sv, sm = inputs.unit_square()
    st, hs = _host_mesh(lib, sv, sm, 2)
    assert lib.elm_mesh_set_annulus(hs, 0.5, 1.5, 6, 0.0) == _lib.ELM_ERR_TOPOLOGY
    cv, cm = inputs.unit_cube()
    st, hc = _host_mesh(lib, cv, cm, 1)
    assert lib.elm_mesh_set_annulus(hc, 0.5, 1.5, 6, 0.0) == _lib.ELM_ERR_ARG      # 2D only
