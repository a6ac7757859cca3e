"""GPU adjoint (elm_advect_adjoint) against the oracle and against the GPU
forward step: transpose interpolation (oracle transpose, dot-product
identity), velocity sensitivity (oracle forward-mode derivative, central
differences on P2-exact fields), determinism, and the autograd wrapper with
step checkpointing."""
import numpy as np
import pytest
import torch

import oracle
from _helpers import match_nodes
from paper_2103_02388_gb300 import _lib, autograd, elm, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-12, "fp32": 1e-5}


# the same 17^3 node lattice for both element orders
LEVEL = {2: 3, 1: 4}


class Pair:
    def __init__(self, level, precision, mesh="cube", order=2):
        v, m = inputs.unit_cube() if mesh == "cube" else inputs.unit_square()
        self.om = oracle.OracleMesh(v, m, level, order=order)
        self.gm = elm.Mesh(v, m, level, precision, adjoint=True, order=order)
        self.order = order
        self.perm = match_nodes(self.om.coords, self.gm.unique_coords())
        self.x = self.om.coords
        self.precision = precision
        umap = self.gm.unique_map()
        first = np.full(self.gm.n_unique, -1, np.int64)
        first[umap[::-1]] = np.arange(self.gm.n_nodes)[::-1]
        self.owner_slot = first          # unique id (GPU order) -> owner slot

    def rounded(self, a):
        return a.astype(np.float32).astype(np.float64) if self.precision == "fp32" else a

    def to_gpu(self, a):
        """Unique field (oracle order) -> storage tensor, copies everywhere."""
        g = np.empty_like(a)
        g[self.perm] = a
        return self.gm.to_storage(torch.tensor(g, dtype=self.gm.dtype, device="cuda"))

    def to_gpu_owner(self, a):
        """Unique field (oracle order) -> storage tensor on owner slots only
        (a gradient of a loss over unique nodes)."""
        g = np.empty_like(a)
        g[self.perm] = a
        out = np.zeros((self.gm.n_nodes,) + a.shape[1:])
        out[self.owner_slot] = g
        return torch.tensor(out, dtype=self.gm.dtype, device="cuda")

    def from_gpu(self, t):
        return self.gm.to_unique(t).double().cpu().numpy()[self.perm]


def _fields(P, kind):
    x = P.x
    if kind == "linear":
        rng = np.random.default_rng(2)
        u = inputs.linear_field(x, rng.standard_normal((3, 3)), np.full(3, 0.5))
        T = inputs.random_quadratic(x, seed=6)
    else:
        u = inputs.random_fourier(x, seed=9) + 0.2 * inputs.uniform_field(x, [0.31, -0.17, 0.23])
        T = inputs.gaussian(x, (0.45, 0.5, 0.55), 0.15)
    return P.rounded(u), P.rounded(T)


@pytest.mark.parametrize("order", [2, 1])
@pytest.mark.parametrize("precision,n_sub", [("fp64", 1), ("fp64", 3), ("fp32", 1)])
def test_transpose_matches_oracle(precision, n_sub, order):
    P = Pair(LEVEL[order], precision, order=order)
    u, T = _fields(P, "fourier")
    dt = inputs.dt_for_cfl(4.0, 3, u)
    g = np.random.default_rng(1).standard_normal(P.om.n_nodes)
    P.gm.set_velocity(P.to_gpu(u))
    gT_old, _, _ = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(g), dt, n_sub)
    P.gm.status()
    got = P.from_gpu(gT_old)
    ref = P.om.advect_transpose(g, u, dt, n_sub)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max() * 10
    # duplicated slots carry no gradient
    umap = P.gm.unique_map()
    ghosts = np.ones(P.gm.n_nodes, bool)
    ghosts[P.owner_slot] = False
    assert np.all(gT_old.cpu().numpy()[ghosts] == 0)


@pytest.mark.parametrize("order", [2, 1])
def test_dot_product_identity_on_gpu(order):
    P = Pair(LEVEL[order], "fp64", order=order)
    u, T = _fields(P, "fourier")
    dt = inputs.dt_for_cfl(4.0, 3, u)
    rng = np.random.default_rng(4)
    a, b = rng.standard_normal(P.om.n_nodes), rng.standard_normal(P.om.n_nodes)
    P.gm.set_velocity(P.to_gpu(u))
    Wa = P.from_gpu(P.gm.advect(P.to_gpu(a), dt, 2))
    WTb, _, _ = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(b), dt, 2)
    lhs, rhs = Wa @ b, a @ P.from_gpu(WTb)
    assert abs(lhs - rhs) <= 1e-12 * np.abs(a).sum() * np.abs(b).max()


@pytest.mark.parametrize("kind,n_sub,order", [("linear", 1, 2), ("linear", 2, 2), ("fourier", 1, 2), ("fourier", 2, 2),
                                              ("linear", 2, 1), ("fourier", 1, 1), ("fourier", 2, 1)])
def test_velocity_gradient_matches_oracle_jvp(kind, n_sub, order):
    """<dL/du, v> from the GPU adjoint equals <g, dT/d eps> of the oracle's
    forward-mode derivative for 8 random directions v (L = <g, T_new>)."""
    P = Pair(LEVEL[order], "fp64", order=order)
    u, T = _fields(P, kind)
    dt = inputs.dt_for_cfl(3.0, 3, u)
    rng = np.random.default_rng(5)
    g = rng.standard_normal(P.om.n_nodes)
    P.gm.set_velocity(P.to_gpu(u))
    _, gU, _ = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(g), dt, n_sub)
    gU = P.from_gpu(gU)
    for _ in range(8):
        v = rng.standard_normal(u.shape)
        _, jvp = P.om.advect_jvp(T, u, v, dt, n_sub)
        lhs, rhs = (gU * v).sum(), g @ jvp
        assert abs(lhs - rhs) <= 1e-9 * (np.abs(g) @ np.abs(jvp) + 1e-30)


@pytest.mark.parametrize("order", [2, 1])
def test_velocity_gradient_time_dependent_split(order):
    P = Pair(LEVEL[order], "fp64", order=order)
    rng = np.random.default_rng(8)
    u0, T = _fields(P, "fourier")
    # a generic shift: no stage point runs exactly along a face of the box
    # (where the clamp makes the step non-differentiable)
    u1 = inputs.random_fourier(P.x, seed=12) + 0.2 * inputs.uniform_field(P.x, [-0.21, 0.33, 0.14])
    dt = inputs.dt_for_cfl(3.0, 3, u1)
    g = rng.standard_normal(P.om.n_nodes)
    P.gm.set_velocity(P.to_gpu(u0), P.to_gpu(u1))
    _, gU0, gU1 = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(g), dt, 2)
    gU0, gU1 = P.from_gpu(gU0), P.from_gpu(gU1)
    zero = np.zeros_like(u0)
    for _ in range(4):
        v = rng.standard_normal(u0.shape)
        _, j0 = P.om.advect_jvp(T, u0, v, dt, 2, u_new=u1, du_new=zero)
        _, j1 = P.om.advect_jvp(T, u0, zero, dt, 2, u_new=u1, du_new=v)
        assert abs((gU0 * v).sum() - g @ j0) <= 1e-9 * (np.abs(g) @ np.abs(j0) + 1e-30)
        assert abs((gU1 * v).sum() - g @ j1) <= 1e-9 * (np.abs(g) @ np.abs(j1) + 1e-30)


@pytest.mark.parametrize("order", [2, 1])
def test_velocity_gradient_finite_differences_gpu(order):
    """Central differences of the GPU forward step on fields the elements
    represent exactly (linear u; quadratic T for P2, linear T for P1)."""
    P = Pair(LEVEL[order], "fp64", order=order)
    u, T = _fields(P, "linear")
    if order == 1:
        T = P.x @ np.array([0.3, -0.2, 0.5]) + 0.1
    dt = 0.04
    rng = np.random.default_rng(3)
    g = rng.standard_normal(P.om.n_nodes)
    inner = np.linalg.norm(P.x - 0.5, axis=1) < 0.3
    g[~inner] = 0.0                          # away from the box clamp
    Tg = P.to_gpu(T)
    P.gm.set_velocity(P.to_gpu(u))
    _, gU, _ = P.gm.advect_adjoint(Tg, P.to_gpu_owner(g), dt, 1)
    gU = P.from_gpu(gU)
    for _ in range(4):
        B = rng.standard_normal((3, 3))
        v = inputs.linear_field(P.x, B, np.full(3, 0.5))
        e = 1e-6
        P.gm.set_velocity(P.to_gpu(u + e * v))
        fp = P.from_gpu(P.gm.advect(Tg, dt, 1))
        P.gm.set_velocity(P.to_gpu(u - e * v))
        fm = P.from_gpu(P.gm.advect(Tg, dt, 1))
        fd = g @ (fp - fm) / (2 * e)
        assert abs((gU * v).sum() - fd) <= 1e-7 * (np.abs(g) @ np.abs((fp - fm) / (2 * e)) + 1e-30)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_convergent_flow_sums_exactly(precision):
    """Every departure point clamped onto one corner node: a uniform velocity
    toward the corner (1, 1, 1) traced back past it, so all 274,625 nodes of
    the level-5 cube send phi = 1 times g_i = 1 to that node.  The sum must be
    exactly n_unique (a fixed-point scale taken from the largest contribution
    alone, with a few bits of headroom, would wrap around), every other entry
    0, and no velocity gradient passes the clamp."""
    P = Pair(5, precision)
    n = P.om.n_nodes
    u = inputs.uniform_field(P.x, [-2.0, -2.0, -2.0])
    T = inputs.gaussian(P.x, (0.5, 0.5, 0.5), 0.2)
    P.gm.set_velocity(P.to_gpu(u))
    gT, gU, _ = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(np.ones(n)), 1.0, 1)
    P.gm.status()
    got = P.from_gpu(gT)
    corner = int(np.argmin(np.abs(P.x - 1.0).sum(axis=1)))
    assert got[corner] == float(n)
    assert np.count_nonzero(got) == 1
    assert not torch.any(gU != 0)
    assert np.array_equal(got, P.om.advect_transpose(np.ones(n), u, 1.0, 1))


def test_small_gradient_entries_keep_relative_precision():
    """dL/dT^n entries spanning twelve decades: g_i = 2^(-40 x1_i), smooth,
    so the few departure points that reach a node (CFL 0.5) carry g of one
    size, and P1 elements, so every contribution phi_j g_i >= 0.  Each entry
    matches the oracle transpose to 1e-12 of itself, not of the largest
    entry (one fixed-point quantum of 2^-52 times the largest contribution
    would already miss this for every entry below 2e-4 of the largest).  The
    check covers the entries whose basis weights are not tiny (sum of phi of
    at least 1e-3): for those, the two implementations' independent roundoff
    in phi stays far below 1e-12 of the entry."""
    P = Pair(LEVEL[1], "fp64", order=1)
    u, T = _fields(P, "fourier")
    dt = inputs.dt_for_cfl(0.5, LEVEL[1], u)
    env = 2.0 ** (-40.0 * P.x[:, 0])
    P.gm.set_velocity(P.to_gpu(u))
    gT, _, _ = P.gm.advect_adjoint(P.to_gpu(T), P.to_gpu_owner(env), dt, 2)
    P.gm.status()
    got, ref = P.from_gpu(gT), P.om.advect_transpose(env, u, dt, 2)
    weight = P.om.advect_transpose(np.ones(P.om.n_nodes), u, dt, 2)   # sum of phi per node
    assert np.all((ref > 0) == (got > 0))
    check = weight >= 1e-3
    assert check.mean() > 0.95
    assert ref[check].min() < 1e-11 * ref.max()       # the entries span many decades
    assert np.all(np.abs(got[check] - ref[check]) <= 1e-12 * ref[check])


def _kink_nodes(P, u, dt, idx, tol=1e-9):
    """Nodes idx (one RK4 substep of dt) with a stage point or departure point
    within tol lattice cells of a micro-element face of the unit cube's
    Freudenthal lattice: a cell fraction near 0 or 1, or two fractions equal
    (the Kuhn planes inside a cell).  Stage points from the oracle's own
    field evaluation."""
    N = 2 ** P.gm.level
    xs = P.x[idx]
    clamp = lambda p: np.clip(p, 0.0, 1.0)  # noqa: E731
    k1 = u[idx]
    z2 = clamp(xs - dt / 2 * k1)
    k2 = P.om.eval(u, z2)
    z3 = clamp(xs - dt / 2 * k2)
    k3 = P.om.eval(u, z3)
    z4 = clamp(xs - dt * k3)
    k4 = P.om.eval(u, z4)
    X = clamp(xs - dt / 6 * (k1 + 2 * k2 + 2 * k3 + k4))
    flag = np.zeros(len(idx), bool)
    for p in (z2, z3, z4, X):
        f = p * N - np.floor(p * N)
        flag |= np.any((f < tol) | (f > 1 - tol), axis=1)
        for a in range(3):
            for b in range(a + 1, 3):
                flag |= np.abs(f[:, a] - f[:, b]) < tol
    return flag


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_config5_level6_velocity_gradient(precision):
    """Config 5's setting at its own size (unit cube, level 6, cellular flow,
    Gaussian T^n, CFL 4): L = <g, T^{n+1}> with g on sampled nodes (four runs
    of 400 nodes; the nodes whose trace runs along a kink are flagged and
    left out).  <dL/du, v> from the GPU adjoint equals the oracle's
    forward-mode derivative on those nodes for 32 random directions v (FP64
    1e-9, FP32 1e-4 relative to sum |g| |dT/d eps|); in FP64 it also matches
    central differences of the GPU step for 8 of them (at most one direction
    may straddle a micro-element face, where the step is only C0)."""
    P = Pair(6, precision)
    n = P.om.n_nodes
    u = P.rounded(inputs.cellular_flow(P.x))
    T = P.rounded(inputs.gaussian(P.x, (0.35, 0.5, 0.5), 0.1))
    dt = inputs.dt_for_cfl(4.0, 6, u)
    rng = np.random.default_rng(21)
    runs = [(400 * b, 400 * b + 400) for b in sorted(rng.choice(n // 400, 4, replace=False))]
    g = np.zeros(n)
    for b, e in runs:
        g[b:e] = rng.standard_normal(e - b)
    # Flagged and left out: nodes whose trace runs along a kink of the step
    # (the step is only C0 there, and the offset form of the GPU and the
    # absolute coordinates of the oracle may round to different one-sided
    # derivatives, both valid): the box boundary, where the cellular flow is
    # tangential only up to rounding (sin(pi) != 0), and every node with an
    # RK4 stage point or departure point on a micro-element face (the flow's
    # symmetries keep whole traces on the planes x = 1/2, y = 1/2 and on
    # diagonal Kuhn planes).
    idx = np.nonzero(g)[0]
    flag = _kink_nodes(P, u, dt, idx) | np.any((P.x[idx] == 0.0) | (P.x[idx] == 1.0), axis=1)
    assert flag.mean() < 0.1
    g[idx[flag]] = 0.0
    Tg = P.to_gpu(T)
    P.gm.set_velocity(P.to_gpu(u))
    _, gU, _ = P.gm.advect_adjoint(Tg, P.to_gpu_owner(g), dt, 1)
    P.gm.status()
    gU = P.from_gpu(gU)
    tol = 1e-9 if precision == "fp64" else 1e-4
    dirs = [rng.standard_normal(u.shape) for _ in range(32)]
    for v in dirs:
        lhs, rhs, scale = (gU * v).sum(), 0.0, 0.0
        for b, e in runs:
            _, jvp = P.om.advect_jvp(T, u, v, dt, 1, begin=b, end=e)
            rhs += g[b:e] @ jvp
            scale += np.abs(g[b:e]) @ np.abs(jvp)
        assert abs(lhs - rhs) <= tol * scale
    if precision != "fp64":
        return
    eps, bad = 1e-6, 0
    for v in dirs[:8]:
        P.gm.set_velocity(P.to_gpu(u + eps * v))
        fp = P.from_gpu(P.gm.advect(Tg, dt, 1))
        P.gm.set_velocity(P.to_gpu(u - eps * v))
        fm = P.from_gpu(P.gm.advect(Tg, dt, 1))
        dT = (fp - fm) / (2 * eps)
        if abs((gU * v).sum() - g @ dT) > 1e-6 * (np.abs(g) @ np.abs(dT)):
            bad += 1
    assert bad <= 1


def test_adjoint_substep_limit():
    P = Pair(2, "fp64")
    u, T = _fields(P, "linear")
    P.gm.set_velocity(P.to_gpu(u))
    g = P.to_gpu_owner(np.ones(P.om.n_nodes))
    with pytest.raises(_lib.ElmError):
        P.gm.advect_adjoint(P.to_gpu(T), g, 0.01, 65)    # above ELM_MAX_ADJOINT_SUBSTEPS


def test_adjoint_is_deterministic():
    P = Pair(3, "fp32")
    u, T = _fields(P, "fourier")
    dt = inputs.dt_for_cfl(6.0, 3, u)
    g = P.to_gpu_owner(np.random.default_rng(2).standard_normal(P.om.n_nodes))
    P.gm.set_velocity(P.to_gpu(u))
    r1 = P.gm.advect_adjoint(P.to_gpu(T), g, dt, 2)
    r2 = P.gm.advect_adjoint(P.to_gpu(T), g, dt, 2)
    assert torch.equal(r1[0], r2[0]) and torch.equal(r1[1], r2[1])


def test_autograd_rollout_with_checkpoints():
    """L = 1/2 |T_K - T*|^2 after K steps: gradients with and without step
    checkpointing agree, and match central differences along a direction of
    T^0 (the map is linear in T^0) and the oracle chain for the velocity."""
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, 3, "fp64", adjoint=True)
    x = mesh.node_coords()
    u = torch.tensor(inputs.random_fourier(x, seed=5), dtype=torch.float64, device="cuda")
    T0 = torch.tensor(inputs.gaussian(x, (0.4, 0.5, 0.5), 0.15), dtype=torch.float64, device="cuda")
    target = torch.tensor(inputs.smooth_target(x, seed=5), dtype=torch.float64, device="cuda")
    dt = inputs.dt_for_cfl(2.0, 3, u.cpu().numpy())
    steps = 12

    def loss(T0_, u_, every):
        T = autograd.rollout(T0_, u_, mesh, dt, steps, checkpoint_every=every)
        return 0.5 * ((T - target) ** 2).sum()

    grads = []
    for every in (0, 4):
        a = T0.clone().requires_grad_(True)
        b = u.clone().requires_grad_(True)
        loss(a, b, every).backward()
        grads.append((a.grad.clone(), b.grad.clone()))
    assert torch.equal(grads[0][0], grads[1][0]) and torch.equal(grads[0][1], grads[1][1])
    gT0 = grads[0][0]
    e = 1e-4
    # the gradient sits on owner slots, so compare along a direction that is
    # equal on all storage copies of a node (as every physical field is)
    mesh_umap = torch.tensor(mesh.unique_map(), device="cuda")
    d_unique = torch.randn(mesh.n_unique, dtype=torch.float64, device="cuda")
    d = d_unique[mesh_umap]
    with torch.no_grad():
        fd = (loss(T0 + e * d, u, 0) - loss(T0 - e * d, u, 0)) / (2 * e)
    assert abs(float((gT0 * d).sum()) - float(fd)) <= 1e-8 * abs(float(fd)) + 1e-10
