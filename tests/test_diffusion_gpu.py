"""GPU parity of the diffusion step (Eq. linear system: Theta scheme, P1 / P2
mass and stiffness, Dirichlet boundary, Jacobi-preconditioned CG) and of the
Strang splitting (Algorithm 2) against the CPU oracle (sparse direct solve),
through the C ABI.

FP64: the CG tolerance is 1e-12 relative; the solution is compared to 1e-10
of max |c|.  FP32: rtol 2e-6, compared to 2e-5 of max |c|.
"""
import numpy as np
import pytest
import torch

import oracle
from _helpers import match_nodes, mesh_for
from paper_2103_02388_gb300 import _lib, elm, inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 2e-5}
RTOL = {"fp64": 1e-12, "fp32": 2e-6}


class Pair:
    def __init__(self, mesh, level, precision="fp64", order=2):
        v, m = mesh_for(mesh) if isinstance(mesh, str) else mesh
        self.om = oracle.OracleMesh(v, m, level, order=order)
        self.gm = elm.Mesh(v, m, level, precision, order=order, diffusion=True)
        self.perm = match_nodes(self.om.coords, self.gm.unique_coords())
        self.precision = precision
        self.x = self.om.coords

    def rounded(self, a):
        return a.astype(np.float32).astype(np.float64) if self.precision == "fp32" else a

    def to_gpu(self, a):
        g = np.empty_like(a)
        g[self.perm] = a
        return self.gm.to_storage(torch.tensor(g, dtype=self.gm.dtype, device="cuda"))

    def from_gpu(self, t):
        return self.gm.to_unique(t).double().cpu().numpy()[self.perm]


def _gauss(x, c, s):
    return np.exp(-np.sum((x - np.asarray(c)) ** 2, axis=1) / (2 * s * s))


@pytest.mark.parametrize("mesh,level,order,precision,theta", [
    ("square", 5, 2, "fp64", 1.0),
    ("square_block", 3, 2, "fp64", 0.5),
    ("cube", 3, 2, "fp64", 1.0),
    ("cube_block", 2, 2, "fp64", 0.5),
    ("cube", 4, 1, "fp64", 1.0),
    ("square", 6, 1, "fp64", 0.5),
    ("cube", 3, 2, "fp32", 1.0),
    ("square", 6, 2, "fp32", 0.5),
    ("cube_block", 2, 1, "fp32", 1.0),
])
def test_diffusion_parity(mesh, level, order, precision, theta):
    P = Pair(mesh, level, precision, order)
    dim = P.x.shape[1]
    c_hat = P.rounded(_gauss(P.x, (0.4, 0.55, 0.5)[:dim], 0.12) + 0.2 * P.x[:, 0])
    c_bnd = P.rounded(0.1 + 0.3 * P.x[:, 1])
    q = P.rounded(np.cos(3.0 * P.x[:, 0]))
    tau, kappa = 0.05, 0.02
    out, it, res = P.gm.diffusion_step(P.to_gpu(c_hat), tau, kappa, theta, c_bnd=P.to_gpu(c_bnd), q=P.to_gpu(q),
                                       rtol=RTOL[precision])
    got = P.from_gpu(out)
    ref = P.om.diffusion_step(c_hat, tau, kappa, theta, c_bnd=c_bnd, q_new=q, q_old=q)
    assert it > 0 and res <= RTOL[precision]
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
    # every storage copy of a node holds the node's value
    umap = torch.tensor(P.gm.unique_map(), device="cuda")
    assert torch.equal(P.gm.to_unique(out)[umap], out)


@pytest.mark.parametrize("dim,order", [(3, 2), (2, 2), (3, 1)])
def test_diffusion_reproduces_fields_in_the_space(dim, order):
    """Manufactured solution (as for the oracle): u in the space, c_hat =
    u - tau kappa Delta u, boundary values u: the discrete solution is u."""
    P = Pair("cube_block" if dim == 3 else "square_block", 2, "fp64", order)
    x = P.x
    if order == 2:
        u = 0.3 + x[:, 0] ** 2 - 2.0 * x[:, 0] * x[:, 1] + 0.5 * x[:, 1] ** 2 + 0.2 * x[:, 0]
        lap = 3.0
    else:
        u = 0.3 + 0.7 * x[:, 0] - 0.4 * x[:, 1]
        lap = 0.0
    tau, kappa = 0.05, 0.3
    out, _, _ = P.gm.diffusion_step(P.to_gpu(u - tau * kappa * lap), tau, kappa, 1.0, c_bnd=P.to_gpu(u), rtol=1e-13)
    assert np.abs(P.from_gpu(out) - u).max() < 1e-11


def _rotating_heat(x, t, kappa):
    """Exact solution of dc/dt + u . grad c = kappa Delta c for the rotation
    u = (0.5 - y, x - 0.5) about the centre of the square: the heat kernel
    (as in the advection-diffusion benchmark of Sec. 3.4) centred at the
    rotated position of (0.5, 0.75)."""
    xc = np.array([0.5 - 0.25 * np.sin(t), 0.5 + 0.25 * np.cos(t)])
    return np.exp(-np.sum((x - xc) ** 2, axis=1) / (4.0 * t * kappa)) / (4.0 * np.pi * t * kappa)


def test_strang_splitting_matches_oracle_and_analytic():
    """Algorithm 2 (diffusion tau/2, advection tau, diffusion tau/2) for a
    diffusing hill carried by the rotation: the GPU follows the oracle's
    composed scheme step by step (1e-10), and both stay close to the exact
    solution (relative H0 error below 1% after a quarter revolution)."""
    P = Pair("square", 5, "fp64", 2)
    kappa = 1e-3
    t0 = 2 * np.pi * 1e-3 / kappa
    steps, T = 20, 0.5 * np.pi
    tau = T / steps
    u = inputs.rotation_2d(P.x, omega=1.0)
    P.gm.set_velocity(P.to_gpu(u))
    c = _rotating_heat(P.x, t0, kappa)
    cg = P.to_gpu(c)
    co = c.copy()
    for k in range(steps):
        t = t0 + k * tau
        bh = _rotating_heat(P.x, t + 0.5 * tau, kappa)
        b1 = _rotating_heat(P.x, t + tau, kappa)
        cg = P.gm.strang_step(cg, tau, kappa, n_sub=1, c_bnd=P.to_gpu(b1), c_bnd_half=P.to_gpu(bh), rtol=1e-12)
        co = P.om.diffusion_step(co, 0.5 * tau, kappa, 1.0, c_bnd=bh)
        co = P.om.advect(co, u, tau)
        co = P.om.diffusion_step(co, 0.5 * tau, kappa, 1.0, c_bnd=b1)
    got = P.from_gpu(cg)
    assert np.abs(got - co).max() <= 1e-10 * np.abs(co).max()
    exact = _rotating_heat(P.x, t0 + T, kappa)
    e = got - exact
    assert np.sqrt(P.om.mass_product(e)) / np.sqrt(P.om.mass_product(exact)) < 0.01


@pytest.mark.parametrize("mesh,level,order,precision", [
    ("triangle", 3, 2, "fp64"),   # one macro: interior stencil only, no shared-face rows
    ("triangle", 4, 1, "fp32"),
    ("cube", 0, 2, "fp64"),       # shared-face rows only, no interior node
    ("cube", 1, 2, "fp32"),
    ("square", 1, 1, "fp64"),     # a single interior unknown, on the shared diagonal
    ("cube", 0, 1, "fp64"),       # no interior unknown at all: nothing to solve
])
def test_diffusion_degenerate_layouts(mesh, level, order, precision):
    """Meshes whose operator has no shared-face rows (the interior stencil
    completes each CG reduction), no interior stencil rows (the face rows do),
    or no interior unknowns, against the oracle."""
    mesh_vm = (np.array([[0.0, 0.0], [1.0, 0.0], [0.2, 0.9]]), np.array([[0, 1, 2]])) if mesh == "triangle" else mesh
    P = Pair(mesh_vm, level, precision, order)
    dim = P.x.shape[1]
    c_hat = P.rounded(_gauss(P.x, (0.4, 0.45, 0.5)[:dim], 0.3) + 0.1 * P.x[:, 0])
    c_bnd = P.rounded(0.2 + 0.1 * P.x[:, 1])
    tau, kappa = 0.05, 0.05
    out, it, res = P.gm.diffusion_step(P.to_gpu(c_hat), tau, kappa, 1.0, c_bnd=P.to_gpu(c_bnd),
                                       rtol=RTOL[precision])
    got = P.from_gpu(out)
    ref = P.om.diffusion_step(c_hat, tau, kappa, 1.0, c_bnd=c_bnd)
    assert np.abs(got - ref).max() <= TOL[precision] * np.abs(ref).max()
    if mesh == "cube" and level == 0 and order == 1:
        assert it == 0
    else:
        assert it > 0 and res <= RTOL[precision]


def test_diffusion_errors():
    v, m = inputs.unit_cube()
    plain = elm.Mesh(v, m, 2, "fp64")
    c = torch.ones(plain.n_nodes, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.ElmError) as e:
        plain.diffusion_step(c, 0.1, 0.1)
    assert e.value.status == _lib.ELM_ERR_STATE
    gm = elm.Mesh(v, m, 3, "fp64", diffusion=True)
    x = torch.tensor(gm.node_coords(), device="cuda")
    c = torch.sin(3.0 * x[:, 0]) * torch.cos(2.0 * x[:, 1])
    with pytest.raises(_lib.ElmError) as e:
        gm.diffusion_step(c, 0.1, 1.0, max_iter=1, rtol=1e-14)
    assert e.value.status == _lib.ELM_ERR_NOT_CONVERGED
    with pytest.raises(_lib.ElmError) as e:
        gm.diffusion_step(c, 0.1, 1.0, out=c)
    assert e.value.status == _lib.ELM_ERR_ARG
    with pytest.raises(_lib.ElmError):
        gm.diffusion_step(c, -0.1, 1.0)
    with pytest.raises(_lib.ElmError):
        gm.diffusion_step(c, 0.1, 1.0, theta=1.5)
    # kappa = 0 (or tau = 0): the mass matrix alone, c_new = c_hat
    out, _, _ = gm.diffusion_step(c, 0.1, 0.0)
    assert torch.allclose(out, c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("case", ["cube-p2-fp64", "cube-p2-fp32", "cube-p1-fp32", "square-p2-fp64", "annulus-p2-fp64"])
def test_diffusion_is_deterministic(case):
    """The operator adds every element contribution in a fixed order (colour
    passes and an ordered fold, no atomics), so repeated solves of one
    system give bitwise the same result and the same iteration count."""
    kind, p, prec = case.split("-")
    order = int(p[1])
    if kind == "annulus":
        v, m = inputs.annulus_ring(6, 2)
        mesh = elm.Mesh(v, m, 4, prec, order=order, diffusion=True, annulus=(0.5, 1.5, 6, 0.0))
    else:
        v, m = inputs.unit_cube() if kind == "cube" else inputs.unit_square()
        mesh = elm.Mesh(v, m, 4 if kind == "cube" else 6, prec, order=order, diffusion=True)
    x = mesh.node_coords()
    c = torch.tensor(np.exp(-((x - 0.4) ** 2).sum(1) / 0.05) + 0.3 * x[:, 0], dtype=mesh.dtype, device="cuda")
    rtol = 1e-11 if prec == "fp64" else 1e-5
    outs = [mesh.diffusion_step(c, 0.01, 0.05, 1.0, rtol=rtol) for _ in range(3)]
    for o in outs[1:]:
        assert torch.equal(o[0], outs[0][0])
        assert o[1] == outs[0][1]
