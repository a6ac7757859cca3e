"""CPU oracle for the MMOC advection step -- TEST INFRASTRUCTURE ONLY.

A plain FP64 C++ restatement (``elm_oracle.cpp``) of the advection step of
Kohl et al., "A massively parallel Eulerian-Lagrangian method for
advection-dominated transport in viscous fluids" (arXiv 2103.02388): Sec. 2.3.1
steps (i)-(iii), Eq. (departure point) integrated by classic RK4, the time
interpolation of Eq. (linear interpolation), the field evaluation of Sec. 2.3.2
with P1 or P2 elements (Sec. 3.1), traces continued over several time steps
(look-back distance, Sec. 2.3.3) and the mass-matrix metrics of Sec. 3.1.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  It shares no code with the CUDA
library in ``paper_2103_02388_gb300``; the two meet only through the seeded
input arrays of ``paper_2103_02388_gb300.inputs``.

Every function either has a pin in ``tests/test_oracle_*.py`` (values fixed by
the mathematics or printed in the paper) or is marked "parity unpinned" below.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "elm_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compiles the oracle with the host C++ compiler; returns the library path."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-pthread",
                               _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        lib.orc_mesh_create.restype = P
        lib.orc_mesh_create.argtypes = [I32, I64, P, I64, P, I32, I32]
        lib.orc_mesh_destroy.argtypes = [P]
        lib.orc_num_nodes.restype = I64
        lib.orc_num_nodes.argtypes = [P]
        lib.orc_node_coords.argtypes = [P, P]
        lib.orc_macro_nodes.restype = I64
        lib.orc_macro_nodes.argtypes = [P, I64, P, P]
        lib.orc_locate.argtypes = [P, I64, P, P, P, P]
        lib.orc_eval.argtypes = [P, P, I32, I64, P, P, I32]
        lib.orc_departure.argtypes = [P, P, P, D, I32, I64, I64, P, I32]
        lib.orc_trace.argtypes = [P, P, P, D, I32, I64, P, P, I32]
        lib.orc_advect.argtypes = [P, P, P, P, P, D, I32, I64, I64, I32]
        lib.orc_advect_nodes.argtypes = [P, P, P, P, D, I32, I64, P, P, I32]
        lib.orc_advect_transpose.argtypes = [P, P, P, P, P, D, I32]
        lib.orc_advect_jvp.argtypes = [P, P, P, P, P, P, D, I32, I64, I64, P, P, I32]
        lib.orc_mass_products.argtypes = [P, I32, P, P, P]
        lib.orc_micro_simplices.restype = I64
        lib.orc_micro_simplices.argtypes = [P, P, P]
        lib.orc_mass_unit.argtypes = [I32, I32, P]
        lib.orc_element_matrices.restype = I64
        lib.orc_element_matrices.argtypes = [P, P, P, P]
        lib.orc_boundary_nodes.argtypes = [P, P]
        lib.orc_set_annulus.restype = I32
        lib.orc_set_annulus.argtypes = [P, D, D, I32, D]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def default_threads() -> int:
    return os.cpu_count() or 1


class OracleMesh:
    """Macro mesh refined to ``level`` with its global P2 (``order`` 2) or P1
    (``order`` 1) nodes (Sec. 2.1, 2.2, 3.1).

    ``vertices``: [n_vertices, dim] float64; ``macros``: [n_macros, dim+1]
    vertex ids.  Node numbering is the oracle's own; tests map it onto the CUDA
    library's numbering by coordinates.
    """

    def __init__(self, vertices, macros, level: int, order: int = 2, annulus=None):
        lib = _load()
        self.vertices = _f64(vertices)
        self.macros = np.ascontiguousarray(macros, dtype=np.int64)
        self.dim = int(self.vertices.shape[1])
        self.level = int(level)
        self.order = int(order)
        self._h = lib.orc_mesh_create(self.dim, self.vertices.shape[0], _ptr(self.vertices),
                                      self.macros.shape[0], _ptr(self.macros), self.level, self.order)
        if not self._h:
            raise ValueError("oracle: invalid mesh")
        self.annulus = annulus
        if annulus is not None:
            # (r_min, r_max, n_sectors, theta0): blended onto the annulus (Sec. 2.1)
            rmin, rmax, nsec, th0 = annulus
            if lib.orc_set_annulus(self._h, float(rmin), float(rmax), int(nsec), float(th0)) != 0:
                raise ValueError("oracle: not a 2D ring mesh")
        self.n_nodes = int(lib.orc_num_nodes(self._h))
        self.coords = np.empty((self.n_nodes, self.dim))
        lib.orc_node_coords(self._h, _ptr(self.coords))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().orc_mesh_destroy(h)
            self._h = None

    # -- structure ---------------------------------------------------------
    def macro_nodes(self, macro: int):
        """Lattice coordinates p of the macro's nodes and their node ids."""
        lib = _load()
        n = lib.orc_macro_nodes(self._h, macro, None, None)
        p = np.empty((n, self.dim), np.int32)
        ids = np.empty(n, np.int32)
        lib.orc_macro_nodes(self._h, macro, _ptr(p), _ptr(ids))
        return p, ids

    def micro_simplices(self):
        """All micro simplices: (macro ids [n], vertex lattice points [n, d+1, d])."""
        lib = _load()
        n = lib.orc_micro_simplices(self._h, None, None)
        m = np.empty(n, np.int64)
        w = np.empty((n, self.dim + 1, self.dim), np.int32)
        lib.orc_micro_simplices(self._h, _ptr(m), _ptr(w))
        return m, w

    def locate(self, pts):
        """Box clamp, macro search and O(1) micro location of each point."""
        pts = _f64(pts).reshape(-1, self.dim)
        n = pts.shape[0]
        m = np.empty(n, np.int64)
        w = np.empty((n, self.dim + 1, self.dim), np.int32)
        mu = np.empty((n, self.dim + 1))
        _load().orc_locate(self._h, n, _ptr(pts), _ptr(m), _ptr(w), _ptr(mu))
        return m, w, mu

    # -- field evaluation and the advection step ----------------------------
    def eval(self, field, pts, threads: int | None = None):
        """P1 / P2 interpolant of ``field`` ([n_nodes] or [n_nodes, c]) at ``pts``."""
        field = _f64(field)
        ncomp = 1 if field.ndim == 1 else field.shape[1]
        pts = _f64(pts).reshape(-1, self.dim)
        out = np.empty((pts.shape[0], ncomp))
        _load().orc_eval(self._h, _ptr(field), ncomp, pts.shape[0], _ptr(pts), _ptr(out),
                         threads or default_threads())
        return out[:, 0] if field.ndim == 1 else out

    def departure(self, u_old, dt, n_sub=1, u_new=None, begin=0, end=None, threads=None):
        """Departure points X(x_i, t_{n+1}, t_n) of nodes [begin, end)."""
        u_old = _f64(u_old)
        u_new = u_old if u_new is None else _f64(u_new)
        end = self.n_nodes if end is None else end
        X = np.empty((end - begin, self.dim))
        _load().orc_departure(self._h, _ptr(u_old), _ptr(u_new), float(dt), int(n_sub),
                              begin, end, _ptr(X), threads or default_threads())
        return X

    def trace(self, X, u_old, dt, n_sub=1, u_new=None, threads=None):
        """Continues backward traces from the points ``X`` ([n, dim]) over one
        further interval of length dt whose velocity is u_old at its start and
        u_new at its end (Sec. 2.3.3); returns the new points."""
        X = _f64(X).reshape(-1, self.dim)
        u_old = _f64(u_old)
        u_new = u_old if u_new is None else _f64(u_new)
        out = np.empty_like(X)
        _load().orc_trace(self._h, _ptr(u_old), _ptr(u_new), float(dt), int(n_sub), X.shape[0],
                          _ptr(X), _ptr(out), threads or default_threads())
        return out

    def advect(self, T_old, u_old, dt, n_sub=1, u_new=None, begin=0, end=None, threads=None):
        """One MMOC advection step: T^{n+1}_i = T^n_h(X_i) for nodes [begin, end)."""
        T_old = _f64(T_old)
        u_old = _f64(u_old)
        u_new = u_old if u_new is None else _f64(u_new)
        end = self.n_nodes if end is None else end
        out = np.empty(end - begin)
        _load().orc_advect(self._h, _ptr(u_old), _ptr(u_new), _ptr(T_old), _ptr(out),
                           float(dt), int(n_sub), begin, end, threads or default_threads())
        return out

    def advect_nodes(self, T_old, u_old, dt, idx, n_sub=1, u_new=None, threads=None):
        """One advection step evaluated only at the node ids ``idx``."""
        T_old = _f64(T_old)
        u_old = _f64(u_old)
        u_new = u_old if u_new is None else _f64(u_new)
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        out = np.empty(idx.shape[0])
        _load().orc_advect_nodes(self._h, _ptr(u_old), _ptr(u_new), _ptr(T_old), float(dt), int(n_sub),
                                 idx.shape[0], _ptr(idx), _ptr(out), threads or default_threads())
        return out

    def advect_jvp(self, T_old, u_old, du_old, dt, n_sub=1, u_new=None, du_new=None, threads=None,
                   begin=0, end=None):
        """(T_new, dT_new/d eps) for u -> u + eps du (forward mode, dual numbers)
        at nodes [begin, end).  For a steady velocity (u_new None) the
        direction is du_old."""
        T_old = _f64(T_old)
        u_old = _f64(u_old)
        du_old = _f64(du_old)
        steady = u_new is None
        u_new = u_old if steady else _f64(u_new)
        du_new = du_old if steady else _f64(du_new)
        end = self.n_nodes if end is None else end
        out = np.empty(end - begin)
        jvp = np.empty(end - begin)
        _load().orc_advect_jvp(self._h, _ptr(u_old), _ptr(u_new), _ptr(du_old), _ptr(du_new), _ptr(T_old),
                               float(dt), int(n_sub), int(begin), int(end), _ptr(out), _ptr(jvp),
                               threads or default_threads())
        return out, jvp

    def advect_transpose(self, g_new, u_old, dt, n_sub=1, u_new=None):
        """Transpose of the advection step's interpolation matrix applied to g_new."""
        g_new = _f64(g_new)
        u_old = _f64(u_old)
        u_new = u_old if u_new is None else _f64(u_new)
        out = np.empty(self.n_nodes)
        _load().orc_advect_transpose(self._h, _ptr(u_old), _ptr(u_new), _ptr(g_new), _ptr(out),
                                     float(dt), int(n_sub))
        return out

    # -- diffusion step (Eq. linear system) ----------------------------------
    def element_matrices(self):
        """(nodes [n_simplices, nb], M_e [n_simplices, nb, nb], A_e [...]) of every
        micro simplex: local mass and stiffness matrices."""
        lib = _load()
        n = int(lib.orc_element_matrices(self._h, None, None, None))
        nb = self.dim + 1 if self.order == 1 else (self.dim + 1) * (self.dim + 2) // 2
        nodes = np.empty((n, nb), np.int32)
        Me = np.empty((n, nb, nb))
        Ae = np.empty((n, nb, nb))
        lib.orc_element_matrices(self._h, _ptr(nodes), _ptr(Me), _ptr(Ae))
        return nodes, Me, Ae

    def assemble(self):
        """Global sparse mass matrix M and stiffness matrix A (scipy CSR)."""
        import scipy.sparse as sp
        nodes, Me, Ae = self.element_matrices()
        nb = nodes.shape[1]
        rows = np.repeat(nodes, nb, axis=1).ravel()
        cols = np.tile(nodes, (1, nb)).ravel()
        shape = (self.n_nodes, self.n_nodes)
        M = sp.coo_matrix((Me.ravel(), (rows, cols)), shape=shape).tocsr()
        A = sp.coo_matrix((Ae.ravel(), (rows, cols)), shape=shape).tocsr()
        return M, A

    def boundary(self):
        """Boolean mask of the nodes on the boundary of the mesh."""
        out = np.empty(self.n_nodes, np.uint8)
        _load().orc_boundary_nodes(self._h, _ptr(out))
        return out.astype(bool)

    def diffusion_step(self, c_hat, tau, kappa, theta=1.0, c_bnd=None, q_old=None, q_new=None):
        """One solve of Eq. (linear system): (M + tau theta kappa A) c =
        (M - tau (1 - theta) kappa A) c_hat + tau (theta q_new + (1 - theta) q_old),
        with c = c_bnd on the boundary nodes (Dirichlet; c_bnd defaults to
        c_hat there).  q_old / q_new are nodal source values (the load vector
        is M q).  Direct sparse solve on the interior nodes."""
        import scipy.sparse.linalg as sla
        M, A = self._ma if getattr(self, "_ma", None) is not None else self.assemble()
        self._ma = (M, A)
        c_hat = _f64(c_hat)
        E = (M + (tau * theta * kappa) * A).tocsr()
        b = M @ c_hat - (tau * (1.0 - theta) * kappa) * (A @ c_hat)
        if q_old is not None or q_new is not None:
            q = theta * (_f64(q_new) if q_new is not None else 0.0) + (1.0 - theta) * (
                _f64(q_old) if q_old is not None else 0.0)
            b = b + tau * (M @ (q * np.ones(self.n_nodes)))
        bnd = self.boundary()
        c = np.empty(self.n_nodes)
        c[bnd] = (c_hat if c_bnd is None else _f64(c_bnd))[bnd]
        inner = ~bnd
        rhs = b[inner] - E[inner][:, bnd] @ c[bnd]
        c[inner] = sla.spsolve(E[inner][:, inner].tocsc(), rhs)
        return c

    # -- metrics (Sec. 3.1) ---------------------------------------------------
    def mass_product(self, a, b=None):
        """a^T M b with the mass matrix M of the mesh's element order."""
        a = _f64(a).reshape(self.n_nodes, 1)
        b = a if b is None else _f64(b).reshape(self.n_nodes, 1)
        out = np.empty(1)
        _load().orc_mass_products(self._h, 1, _ptr(a), _ptr(b), _ptr(out))
        return float(out[0])

    def metrics(self, c_computed, c_exact, c_initial):
        """H0 error, var, E_peak and the relative mass difference of Sec. 3.1."""
        c_computed = _f64(c_computed)
        e = _f64(c_exact) - c_computed
        ones = np.ones(self.n_nodes)
        m_t = self.mass_product(ones, c_computed)
        m_0 = self.mass_product(ones, _f64(c_initial))
        return {
            "h0": float(np.sqrt(max(self.mass_product(e), 0.0))),
            "var": float(c_computed.max() - c_computed.min()),
            "e_peak": float(c_computed.max() / np.max(c_exact) - 1.0),
            "dm": float(m_t / m_0 - 1.0),
        }


def mass_unit(dim: int, order: int = 2) -> np.ndarray:
    """P1 / P2 mass matrix of a simplex with unit volume (P2: vertex basis
    first, then edges)."""
    nb = dim + 1 if order == 1 else (dim + 1) * (dim + 2) // 2
    out = np.empty((nb, nb))
    _load().orc_mass_unit(dim, int(order), _ptr(out))
    return out


def p2_mass_unit(dim: int) -> np.ndarray:
    """P2 mass matrix of a simplex with unit volume (vertex basis first, then edges)."""
    return mass_unit(dim, 2)
