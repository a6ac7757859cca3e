"""Shared test plumbing: node matching between the oracle's and the CUDA
library's numbering, and seeded workloads on both sides."""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from paper_2103_02388_gb300 import inputs


def _lattice_keys(c: np.ndarray, scale: float):
    q = np.rint(c * scale)
    if np.abs(q - c * scale).max() > 1e-6:
        return None
    q = q.astype(np.int64)
    key = np.zeros(len(c), np.int64)
    for k in range(c.shape[1]):
        key = key * (int(scale) + 1) + q[:, k]
    return key


def match_nodes(coords_ref: np.ndarray, coords_other: np.ndarray, tol: float = 1e-9) -> np.ndarray:
    """perm with coords_other[perm[i]] == coords_ref[i] (to ``tol``); bijective."""
    assert coords_ref.shape == coords_other.shape
    # fast path: both node sets on the 1/2048 lattice (every uniform refinement
    # of a unit-box mesh with dyadic vertices up to that resolution)
    ka = _lattice_keys(coords_ref, 2048.0)
    kb = _lattice_keys(coords_other, 2048.0) if ka is not None else None
    if ka is not None and kb is not None:
        oa, ob = np.argsort(ka), np.argsort(kb)
        if np.array_equal(ka[oa], kb[ob]):
            perm = np.empty(len(ka), np.int64)
            perm[oa] = ob
            assert np.abs(coords_other[perm] - coords_ref).max() <= tol
            return perm
    tree = cKDTree(coords_other)
    dist, perm = tree.query(coords_ref, k=1)
    assert dist.max() <= tol, f"unmatched node, distance {dist.max()}"
    assert len(np.unique(perm)) == len(perm), "node matching is not a bijection"
    return perm


def mesh_for(name: str):
    if name == "square":
        return inputs.unit_square()
    if name == "cube":
        return inputs.unit_cube()
    if name == "cube_block":
        return inputs.cube_block(2, perturb=0.25, seed=7)
    if name == "square_block":
        return inputs.square_block(3, perturb=0.25, seed=7)
    raise KeyError(name)


def velocity_for(name: str, coords: np.ndarray, seed: int = 3):
    dim = coords.shape[1]
    if name == "rotation":
        return inputs.rotation_2d(coords) if dim == 2 else inputs.rotation_3d(coords)
    if name == "cellular":
        return inputs.cellular_flow(coords)
    if name == "fourier":
        return inputs.random_fourier(coords, seed=seed)
    if name == "zero":
        return np.zeros_like(coords)
    raise KeyError(name)


def scalar_for(name: str, coords: np.ndarray):
    dim = coords.shape[1]
    if name == "gauss":
        return inputs.gaussian(coords, (0.35, 0.5, 0.5)[:dim] if dim == 3 else (0.25, 0.5), 0.1 if dim == 3 else 0.05)
    if name == "slotted":
        return inputs.slotted_sphere(coords) if dim == 3 else inputs.slotted_cylinder(coords)
    if name == "quadratic":
        return inputs.random_quadratic(coords, seed=5)
    raise KeyError(name)
