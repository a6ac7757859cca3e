"""Seeded synthetic inputs shared by the CUDA path's tests, the oracle's tests
and the benchmark.

This module holds meshes (macro vertex coordinates and macro vertex lists) and
analytic fields sampled at given coordinates.  It contains none of the
advection method's arithmetic (no location, interpolation or integration), so
that both the CUDA library and the CPU oracle can take their inputs from it
without sharing any of the method.

The workloads follow the paper's benchmarks where they are analytic
(Sec. 3.2 circular advection, Table 1 and Table 2), and otherwise the
synthetic recipes of the GB300 benchmark configurations:

* rotation in the unit square on 2 macro triangles, Gaussian cone;
* cellular flow in the unit cube on 6 Kuhn macro tetrahedra, slotted sphere;
* seeded random smooth (curl of Fourier-mode stream functions) velocity,
  Gaussian cone.
"""
from __future__ import annotations

import itertools

import numpy as np

# ---------------------------------------------------------------------------
# Meshes
# ---------------------------------------------------------------------------


def unit_square():
    """Unit square split along the (0,0)-(1,1) diagonal into 2 triangles."""
    v = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0], [1.0, 1.0]])
    macros = np.array([[0, 1, 3], [0, 2, 3]], dtype=np.int64)
    return v, macros


def unit_cube():
    """Unit cube split into the 6 Kuhn tetrahedra 0, e_a, e_a+e_b, 1."""
    v = np.array([[x, y, z] for z in (0.0, 1.0) for y in (0.0, 1.0) for x in (0.0, 1.0)])
    vid = lambda p: int(p[0] + 2 * p[1] + 4 * p[2])  # noqa: E731
    macros = []
    for perm in itertools.permutations(range(3)):
        p = np.zeros(3, dtype=int)
        tet = [vid(p)]
        for a in perm:
            p[a] = 1
            tet.append(vid(p))
        macros.append(tet)
    return v, np.array(macros, dtype=np.int64)


def cube_block(k: int, perturb: float = 0.0, seed: int = 0):
    """[0,1]^3 as a k x k x k block of cubes, 6 Kuhn tetrahedra each.

    ``perturb`` moves every interior vertex by up to ``perturb / k`` in each
    axis (seeded), which gives non-uniform macro shapes while the domain stays
    the unit cube.
    """
    g = np.linspace(0.0, 1.0, k + 1)
    v = np.array([[x, y, z] for z in g for y in g for x in g])
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        inner = np.all((v > 0.0) & (v < 1.0), axis=1)
        v[inner] += rng.uniform(-perturb / k, perturb / k, size=(int(inner.sum()), 3))
    vid = lambda p: int(p[0] + (k + 1) * p[1] + (k + 1) ** 2 * p[2])  # noqa: E731
    macros = []
    for cz, cy, cx in itertools.product(range(k), repeat=3):
        base = np.array([cx, cy, cz])
        for perm in itertools.permutations(range(3)):
            p = base.copy()
            tet = [vid(p)]
            for a in perm:
                p[a] += 1
                tet.append(vid(p))
            macros.append(tet)
    return v, np.array(macros, dtype=np.int64)


def annulus_ring(n_sectors: int = 6, n_layers: int = 2, r_min: float = 0.5, r_max: float = 1.5,
                 theta0: float = 0.0):
    """Coarse ring mesh of an annulus (Sec. 3.4): n_sectors sectors times
    n_layers radial layers, vertices on the circles r_min + (r_max - r_min) j /
    n_layers at the angles theta0 + 2 pi k / n_sectors, two triangles per
    cell.  Blending maps it onto the annulus.  Returns (vertices, triangles)."""
    th = theta0 + 2.0 * np.pi * np.arange(n_sectors) / n_sectors
    radii = r_min + (r_max - r_min) * np.arange(n_layers + 1) / n_layers
    v = np.concatenate([np.stack([r * np.cos(th), r * np.sin(th)], axis=1) for r in radii])
    tris = []
    for j in range(n_layers):
        for k in range(n_sectors):
            k1 = (k + 1) % n_sectors
            a, b = j * n_sectors + k, j * n_sectors + k1
            c, d = (j + 1) * n_sectors + k, (j + 1) * n_sectors + k1
            tris.append([a, b, c])
            tris.append([b, d, c])
    return v, np.array(tris, dtype=np.int64)


def heat_kernel_rotating(x, t: float, kappa: float, start=(0.0, 1.0)):
    """The exact solution of the advection-diffusion benchmark of Sec. 3.4:
    the heat kernel 1/(4 pi t kappa) exp(-r^2 / (4 t kappa)) centred at the
    start point rotated by the angle t about the origin."""
    x = np.asarray(x, dtype=np.float64)
    c = np.array([start[0] * np.cos(t) - start[1] * np.sin(t), start[0] * np.sin(t) + start[1] * np.cos(t)])
    r2 = np.sum((x - c) ** 2, axis=1)
    return np.exp(-r2 / (4.0 * t * kappa)) / (4.0 * np.pi * t * kappa)


def square_block(k: int, perturb: float = 0.0, seed: int = 0):
    """[0,1]^2 as a k x k block of squares, 2 triangles each (diagonal (1,1))."""
    g = np.linspace(0.0, 1.0, k + 1)
    v = np.array([[x, y] for y in g for x in g])
    if perturb > 0.0:
        rng = np.random.default_rng(seed)
        inner = np.all((v > 0.0) & (v < 1.0), axis=1)
        v[inner] += rng.uniform(-perturb / k, perturb / k, size=(int(inner.sum()), 2))
    vid = lambda x, y: int(x + (k + 1) * y)  # noqa: E731
    macros = []
    for cy, cx in itertools.product(range(k), repeat=2):
        macros.append([vid(cx, cy), vid(cx + 1, cy), vid(cx + 1, cy + 1)])
        macros.append([vid(cx, cy), vid(cx, cy + 1), vid(cx + 1, cy + 1)])
    return v, np.array(macros, dtype=np.int64)


def unique_node_count(dim: int, level: int) -> int:
    """Number of P2 nodes of the unit square / cube at ``level``: (2^(L+1)+1)^d."""
    return (2 ** (level + 1) + 1) ** dim


# ---------------------------------------------------------------------------
# Velocity fields (sampled at node coordinates, FP64)
# ---------------------------------------------------------------------------


def rotation_2d(x, omega: float = 2.0 * np.pi, centre=(0.5, 0.5)):
    """Solid-body rotation omega * (c_y - y, x - c_x)."""
    x = np.asarray(x, dtype=np.float64)
    return np.stack([omega * (centre[1] - x[:, 1]), omega * (x[:, 0] - centre[0])], axis=1)


def rotation_3d(x, axis=(1.0, 2.0, 3.0), omega: float = 2.0 * np.pi, centre=(0.5, 0.5, 0.5)):
    """Solid-body rotation omega * a x (x - c) about the unit axis a."""
    x = np.asarray(x, dtype=np.float64)
    a = np.asarray(axis, dtype=np.float64)
    a = a / np.linalg.norm(a)
    return omega * np.cross(a, x - np.asarray(centre))


def linear_field(x, A, centre):
    """u = A (x - c) for a constant matrix A (P1, hence reproduced by P2)."""
    x = np.asarray(x, dtype=np.float64)
    return (x - np.asarray(centre)) @ np.asarray(A, dtype=np.float64).T


def uniform_field(x, u):
    x = np.asarray(x, dtype=np.float64)
    return np.broadcast_to(np.asarray(u, dtype=np.float64), x.shape).copy()


def cellular_flow(x):
    """(sin pi x cos pi y, -cos pi x sin pi y, 0.3 sin pi z)."""
    x = np.asarray(x, dtype=np.float64)
    px, py, pz = np.pi * x[:, 0], np.pi * x[:, 1], np.pi * x[:, 2]
    return np.stack([np.sin(px) * np.cos(py), -np.cos(px) * np.sin(py), 0.3 * np.sin(pz)], axis=1)


def swirl_3d(x, t: float, period: float = 1.5):
    """The time-dependent swirling flow of Sec. 3.3 at time t."""
    x = np.asarray(x, dtype=np.float64)
    g = np.cos(np.pi * t / period)
    s = lambda k, a: np.sin(k * np.pi * x[:, a])  # noqa: E731
    return np.stack([2.0 * s(1, 0) ** 2 * s(2, 1) * s(2, 2) * g,
                     -s(2, 0) * s(1, 1) ** 2 * s(2, 2) * g,
                     -s(2, 0) * s(2, 1) * s(1, 2) ** 2 * g], axis=1)


def random_fourier(x, seed: int, n_modes: int = 8, max_speed: float = 1.0):
    """Divergence-free random smooth velocity: the curl of n_modes stream functions.

    3D mode k: axis a_k in {0,1,2}, integers m, n in {1,2,3}, p in {0,1,2},
    amplitude A_k ~ N(0,1); psi_k = A_k sin(m pi x_b) sin(n pi x_c) cos(p pi x_a)
    with (a, b, c) cyclic, u += curl(psi_k e_a), i.e. u_b += d psi/d x_c,
    u_c -= d psi/d x_b.  2D: psi = A sin(m pi x) sin(n pi y), u = (psi_y, -psi_x).
    The field is scaled so that the maximum speed over the given points is
    ``max_speed``.  u . n = 0 on the unit square / cube boundary.
    """
    x = np.asarray(x, dtype=np.float64)
    dim = x.shape[1]
    rng = np.random.default_rng(seed)
    u = np.zeros_like(x)
    pi = np.pi
    for _ in range(n_modes):
        A = rng.standard_normal()
        m, n = rng.integers(1, 4, size=2)
        if dim == 2:
            # psi = A sin(m pi x) sin(n pi y)
            u[:, 0] += A * np.sin(m * pi * x[:, 0]) * n * pi * np.cos(n * pi * x[:, 1])
            u[:, 1] -= A * m * pi * np.cos(m * pi * x[:, 0]) * np.sin(n * pi * x[:, 1])
            continue
        a = int(rng.integers(0, 3))
        p = int(rng.integers(0, 3))
        b, c = (a + 1) % 3, (a + 2) % 3
        sb, cb = np.sin(m * pi * x[:, b]), np.cos(m * pi * x[:, b])
        sc, cc = np.sin(n * pi * x[:, c]), np.cos(n * pi * x[:, c])
        ca = np.cos(p * pi * x[:, a])
        u[:, b] += A * sb * (n * pi * cc) * ca      # d psi / d x_c
        u[:, c] -= A * (m * pi * cb) * sc * ca      # d psi / d x_b
    speed = np.sqrt((u * u).sum(axis=1)).max()
    return u * (max_speed / speed)


# ---------------------------------------------------------------------------
# Scalar fields
# ---------------------------------------------------------------------------


def gaussian(x, centre, sigma: float):
    x = np.asarray(x, dtype=np.float64)
    r2 = ((x - np.asarray(centre)) ** 2).sum(axis=1)
    return np.exp(-r2 / (2.0 * sigma * sigma))


def slotted_sphere(x, centre=(0.35, 0.5, 0.5), radius: float = 0.15, slot_half: float = 0.025):
    """1 inside the sphere minus the slot {|x - c_x| <= slot_half, y >= c_y}, else 0."""
    x = np.asarray(x, dtype=np.float64)
    c = np.asarray(centre)
    inside = ((x - c) ** 2).sum(axis=1) <= radius * radius
    slot = (np.abs(x[:, 0] - c[0]) <= slot_half) & (x[:, 1] >= c[1])
    return (inside & ~slot).astype(np.float64)


def hill(x, centre=(0.25, 0.5), r0: float = 0.15):
    """The smooth hill of Sec. 3.2: (1 + cos(pi r)) / 4 for r = |x - c| / r0 <= 1."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(((x - np.asarray(centre)) ** 2).sum(axis=1)) / r0
    return np.where(r <= 1.0, 0.25 * (1.0 + np.cos(np.pi * np.minimum(r, 1.0))), 0.0)


def cone(x, centre=(0.5, 0.25), r0: float = 0.15):
    """The cone of Sec. 3.2: 1 - r for r = |x - c| / r0 <= 1."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(((x - np.asarray(centre)) ** 2).sum(axis=1)) / r0
    return np.where(r <= 1.0, 1.0 - r, 0.0)


def slotted_cylinder(x, centre=(0.5, 0.75), r0: float = 0.15):
    """The slotted cylinder of Sec. 3.2 (slot of half width 0.025 below y = 0.85)."""
    x = np.asarray(x, dtype=np.float64)
    r = np.sqrt(((x - np.asarray(centre)) ** 2).sum(axis=1)) / r0
    keep = (np.abs(x[:, 0] - centre[0]) >= 0.025) | (x[:, 1] >= 0.85)
    return ((r <= 1.0) & keep).astype(np.float64)


def three_bodies(x):
    return slotted_cylinder(x) + cone(x) + hill(x)


def half_space(x, cut: float = 0.5):
    """The initial condition of Sec. 3.3: 1 where x_1 < cut, else 0."""
    x = np.asarray(x, dtype=np.float64)
    return (x[:, 0] < cut).astype(np.float64)


def random_linear(x, seed: int):
    """A seeded random affine function a + b . x (in the P1 space exactly)."""
    x = np.asarray(x, dtype=np.float64)
    rng = np.random.default_rng(seed)
    return rng.standard_normal() + x @ rng.standard_normal(x.shape[1])


def random_quadratic(x, seed: int):
    """A seeded random quadratic polynomial q(x) (in the P2 space exactly)."""
    x = np.asarray(x, dtype=np.float64)
    dim = x.shape[1]
    rng = np.random.default_rng(seed)
    c0 = rng.standard_normal()
    g = rng.standard_normal(dim)
    H = rng.standard_normal((dim, dim))
    H = 0.5 * (H + H.T)
    return c0 + x @ g + np.einsum("ni,ij,nj->n", x, H, x)


def smooth_target(x, seed: int):
    """A seeded smooth scalar field (sum of 4 Gaussians), e.g. a loss target."""
    x = np.asarray(x, dtype=np.float64)
    rng = np.random.default_rng(seed)
    out = np.zeros(x.shape[0])
    for _ in range(4):
        c = rng.uniform(0.2, 0.8, size=x.shape[1])
        out += rng.uniform(0.2, 1.0) * gaussian(x, c, rng.uniform(0.05, 0.2))
    return out


# ---------------------------------------------------------------------------
# Time step from a CFL number
# ---------------------------------------------------------------------------


def dt_for_cfl(cfl: float, level: int, u_nodes) -> float:
    """tau = CFL * h_min / max |u| with h_min = 2^-level (unit square / cube)."""
    u = np.asarray(u_nodes, dtype=np.float64)
    vmax = float(np.sqrt((u * u).sum(axis=1)).max())
    return cfl * (0.5 ** level) / vmax


# ---------------------------------------------------------------------------
# Batched workload recipe
# ---------------------------------------------------------------------------


def batch_recipe(seed: int = 4, count: int = 64, levels2d=(4, 5, 6, 7, 8), levels3d=(4, 5, 6)):
    """A seeded list of independent advection instances for the batched form:
    2D unit squares (levels 4-8) and 3D unit cubes (levels 4-6), each with a
    solid-body rotation or a random Fourier velocity (seed 4 + i), a CFL drawn
    from U(0.5, 8), and a Gaussian-cone or slotted scalar."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        dim = 2 if rng.random() < 0.5 else 3
        level = int(rng.choice(levels2d if dim == 2 else levels3d))
        out.append({
            "dim": dim,
            "level": level,
            "velocity": "rotation" if rng.random() < 0.5 else "fourier",
            "velocity_seed": seed + i,
            "cfl": float(rng.uniform(0.5, 8.0)),
            "scalar": "gauss" if rng.random() < 0.5 else "slotted",
        })
    return out


def batch_fields(entry, coords):
    """Velocity and scalar of one batch_recipe entry at the given coordinates."""
    dim = coords.shape[1]
    if entry["velocity"] == "rotation":
        u = rotation_2d(coords) if dim == 2 else rotation_3d(coords)
    else:
        u = random_fourier(coords, seed=entry["velocity_seed"])
    if entry["scalar"] == "gauss":
        T = gaussian(coords, (0.35, 0.5, 0.5)[:dim] if dim == 3 else (0.25, 0.5), 0.1 if dim == 3 else 0.05)
    else:
        T = slotted_sphere(coords) if dim == 3 else slotted_cylinder(coords)
    return u, T, dt_for_cfl(entry["cfl"], entry["level"], u)
