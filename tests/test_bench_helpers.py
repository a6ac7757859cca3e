"""CPU tests of bench.py's host-side helpers: the node matching behind the
full-mesh accuracy record, the traffic record's source hash, and the
workload tables."""
import json

import numpy as np
import pytest

import bench
from paper_2103_02388_gb300 import elm, inputs


@pytest.mark.parametrize("dim,level", [(2, 3), (2, 5), (3, 2), (3, 3)])
def test_match_nodes_pairs_oracle_and_library_nodes(dim, level):
    spec = (dim, level, "fp64", "cellular", "gauss", 4.0, 1)
    om = bench._oracle_mesh(spec)
    v, m = inputs.unit_cube() if dim == 3 else inputs.unit_square()
    gm = elm.Mesh(v, m, level, "fp64", host_only=True)
    uc = gm.unique_coords()
    perm = bench._match_nodes(om.coords, uc, gm.order << gm.level)
    assert np.array_equal(np.sort(perm), np.arange(len(perm)))      # a bijection
    assert np.abs(uc[perm] - om.coords).max() == 0.0                 # same lattice points


def test_match_nodes_rejects_different_node_sets():
    a = np.array([[0.0, 0.0], [0.5, 0.5], [1.0, 1.0]])
    b = np.array([[0.0, 0.0], [0.5, 0.25], [1.0, 1.0]])
    with pytest.raises(RuntimeError):
        bench._match_nodes(a, b, 4)


def test_traffic_record_follows_the_kernel_sources(tmp_path, monkeypatch):
    rec = {"kernel_sha": bench._kernel_hash(), "per_launch_bytes": {"c3-l7-fp32": 123.0}}
    p = tmp_path / "traffic.json"
    p.write_text(json.dumps(rec))
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(p))
    assert bench._traffic("c3-l7-fp32") == 123.0
    assert bench._traffic("c2-l6-fp64") is None          # no figure for that workload
    rec["kernel_sha"] = "0" * 16                          # the sources changed since the capture
    p.write_text(json.dumps(rec))
    assert bench._traffic("c3-l7-fp32") is None


def test_default_workload_is_the_level7_fp32_step():
    assert bench.WORKLOADS["c3-l7-fp32"][:3] == (3, 7, "fp32")
    names = set(bench.WORKLOADS) | set(bench.DIFFUSION_WORKLOADS) | set(bench.VARIANT_WORKLOADS) \
        | set(bench.BATCH_WORKLOADS) | set(bench.ADJOINT_WORKLOADS)
    assert len(names) == len(bench.WORKLOADS) + len(bench.DIFFUSION_WORKLOADS) + len(bench.VARIANT_WORKLOADS) \
        + len(bench.BATCH_WORKLOADS) + len(bench.ADJOINT_WORKLOADS)   # no name shadows another


def test_alg_ops_split_adds_up():
    """The FMA-pipe / ALU-pipe split of the algorithmic operations covers
    every operation of alg_ops_per_node (3D P2 n_sub = 1: 293 + 60 = 353)."""
    import bench
    for dim in (2, 3):
        for n_sub in (1, 2, 4):
            for steady in (True, False):
                fma, alu = bench.alg_ops_split(dim, n_sub, steady)
                assert fma > 0 and alu > 0
                assert fma + alu == bench.alg_ops_per_node(dim, n_sub, steady)
    assert bench.alg_ops_split(3, 1, True) == (293, 60)
