"""Python face of libelm.so: torch tensors in, C-ABI calls out.

Every step of the advection path runs in the library's CUDA kernels; this
module only marshals pointers, sizes and the current CUDA stream.  There is no
CPU fallback: if libelm.so is missing or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import ELM_ADJOINT, ELM_DIFFUSION, ELM_FP32, ELM_FP64, ELM_HOST_ONLY, ELM_HOST_STAGING, ELM_P1, check

_DTYPES = {"fp64": (ELM_FP64, torch.float64, np.float64), "fp32": (ELM_FP32, torch.float32, np.float32)}


def _stream_ptr(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Mesh:
    """A coarse macro mesh refined uniformly to ``level`` (Sec. 2.1).

    ``vertices``: [n_vertices, dim] coordinates; ``macros``: [n_macros, dim+1]
    vertex ids; ``precision``: "fp64" or "fp32"; ``order``: 2 (P2 elements) or
    1 (P1, Sec. 3.1).  ``host_only=True`` builds only the host tables
    (coordinates and the unique map), without a GPU.  ``host_staging=True``
    sets up ``advect_host`` (the step with pinned host buffers).
    """

    def __init__(self, vertices, macros, level: int, precision: str = "fp64", host_only: bool = False,
                 adjoint: bool = False, order: int = 2, diffusion: bool = False, annulus=None,
                 host_staging: bool = False):
        lib = _lib.load()
        self.vertices = np.ascontiguousarray(vertices, dtype=np.float64)
        self.macros = np.ascontiguousarray(macros, dtype=np.int64)
        self.dim = int(self.vertices.shape[1])
        self.level = int(level)
        self.precision = precision
        code, self.dtype, self.np_dtype = _DTYPES[precision]
        self.host_only = host_only
        self.adjoint = adjoint
        if order not in (1, 2):
            raise ValueError("order must be 1 (P1) or 2 (P2)")
        self.order = int(order)
        if not host_only:
            self.device = torch.device("cuda", torch.cuda.current_device())
        h = ctypes.c_void_p()
        check(lib.elm_mesh_create(self.dim, self.vertices.shape[0],
                                  self.vertices.ctypes.data_as(ctypes.c_void_p),
                                  self.macros.shape[0], self.macros.ctypes.data_as(ctypes.c_void_p),
                                  self.level, code | (ELM_HOST_ONLY if host_only else 0) | (ELM_ADJOINT if adjoint else 0)
                                  | (ELM_P1 if order == 1 else 0) | (ELM_DIFFUSION if diffusion else 0)
                                  | (ELM_HOST_STAGING if host_staging else 0),
                                  ctypes.byref(h)))
        self._h = h
        if annulus is not None:
            # (r_min, r_max, n_sectors, theta0): blending onto the annulus (Sec. 2.1)
            r_min, r_max, n_sec, th0 = annulus
            check(lib.elm_mesh_set_annulus(h, float(r_min), float(r_max), int(n_sec), float(th0)))
        self.annulus = annulus
        self.n_nodes = int(lib.elm_mesh_num_nodes(h))
        self.n_unique = int(lib.elm_mesh_num_unique(h))
        self._u = None
        self._host_inflight = []  # (event, host tensors) of advect_host calls not yet complete

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.load().elm_mesh_destroy(h)
            self._h = None

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    # -- host tables ------------------------------------------------------
    def node_coords(self) -> np.ndarray:
        """Coordinates of the storage slots, [n_nodes, dim]."""
        out = np.empty((self.n_nodes, self.dim))
        check(_lib.load().elm_mesh_node_coords(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def unique_map(self) -> np.ndarray:
        """Storage slot -> unique node id, [n_nodes] int64."""
        out = np.empty(self.n_nodes, np.int64)
        check(_lib.load().elm_mesh_unique_map(self._h, out.ctypes.data_as(ctypes.c_void_p)))
        return out

    def unique_coords(self) -> np.ndarray:
        """Coordinates of the unique nodes, [n_unique, dim] (owner slots)."""
        umap = self.unique_map()
        coords = self.node_coords()
        out = np.empty((self.n_unique, self.dim))
        first = np.full(self.n_unique, -1, np.int64)
        slots = np.arange(self.n_nodes)
        first[umap[::-1]] = slots[::-1]
        out[:] = coords[first]
        return out

    # -- layout conversion (device) ---------------------------------------
    def _ncomp(self, t: torch.Tensor, n: int) -> int:
        if t.shape[0] != n:
            raise ValueError(f"expected {n} rows, got {t.shape[0]}")
        return 1 if t.dim() == 1 else int(np.prod(t.shape[1:]))

    def _check_tensor(self, t: torch.Tensor, name: str):
        if not t.is_cuda or t.dtype != self.dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.dtype} CUDA tensor")

    def to_storage(self, t_unique: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._check_tensor(t_unique, "t_unique")
        nc = self._ncomp(t_unique, self.n_unique)
        if out is None:
            out = torch.empty((self.n_nodes,) + tuple(t_unique.shape[1:]), dtype=self.dtype, device=t_unique.device)
        check(_lib.load().elm_to_storage(self._h, ctypes.c_void_p(t_unique.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), nc, _stream_ptr()))
        return out

    def to_unique(self, t_storage: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        self._check_tensor(t_storage, "t_storage")
        nc = self._ncomp(t_storage, self.n_nodes)
        if out is None:
            out = torch.empty((self.n_unique,) + tuple(t_storage.shape[1:]), dtype=self.dtype,
                              device=t_storage.device)
        check(_lib.load().elm_to_unique(self._h, ctypes.c_void_p(t_storage.data_ptr()),
                                        ctypes.c_void_p(out.data_ptr()), nc, _stream_ptr()))
        return out

    # -- the advection step -------------------------------------------------
    def set_velocity(self, u_old: torch.Tensor, u_new: torch.Tensor | None = None) -> None:
        """Borrow the P2 velocity at t_n and t_{n+1} (storage layout, [n, dim])."""
        u_new = u_old if u_new is None else u_new
        for name, u in (("u_old", u_old), ("u_new", u_new)):
            self._check_tensor(u, name)
            if tuple(u.shape) != (self.n_nodes, self.dim):
                raise ValueError(f"{name} must have shape ({self.n_nodes}, {self.dim})")
        check(_lib.load().elm_set_velocity(self._h, ctypes.c_void_p(u_old.data_ptr()),
                                           ctypes.c_void_p(u_new.data_ptr()), _stream_ptr()))
        self._u = (u_old, u_new)  # keep the borrowed buffers alive

    def shift_velocity(self, u_old: torch.Tensor) -> None:
        """Next older look-back interval (Sec. 2.3.3): the current u_old becomes
        u_new (its packed copy is kept) and ``u_old`` ([n, dim], storage
        layout) becomes the new u_old; on the current stream."""
        self._check_tensor(u_old, "u_old")
        if tuple(u_old.shape) != (self.n_nodes, self.dim):
            raise ValueError(f"u_old must have shape ({self.n_nodes}, {self.dim})")
        check(_lib.load().elm_shift_velocity(self._h, ctypes.c_void_p(u_old.data_ptr()), _stream_ptr()))
        self._u = (u_old, self._u[0] if self._u is not None else u_old)

    def advect(self, T_old: torch.Tensor, dt: float, n_sub: int = 1, out: torch.Tensor | None = None,
               stream=None) -> torch.Tensor:
        """One MMOC advection step: T_new[i] = T_old_h(X_i) (storage layout)."""
        self._check_tensor(T_old, "T_old")
        if T_old.shape != (self.n_nodes,):
            raise ValueError(f"T_old must have shape ({self.n_nodes},)")
        if out is None:
            out = torch.empty_like(T_old)
        else:
            self._check_tensor(out, "out")
        check(_lib.load().elm_advect(self._h, ctypes.c_void_p(T_old.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                     float(dt), int(n_sub), _stream_ptr(stream)))
        return out

    def advect_host(self, T_old: torch.Tensor, dt: float, n_sub: int = 1, u_old: torch.Tensor | None = None,
                    u_new: torch.Tensor | None = None, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """The advection step with page-locked HOST tensors (storage layout):
        velocity ``u_old`` ([n, dim], at t_n) and ``u_new`` (at t_{n+1};
        None = steady), ``T_old`` and the result ``out`` ([n]; may be
        ``T_old`` itself).  ``u_old`` None: the mesh's current velocity
        stays resident and only T moves.  Asynchronous on ``stream``: ``out``
        is valid once the stream has completed.  Consecutive calls overlap
        their copies with the previous call's step (mesh created with
        ``host_staging=True``)."""
        if u_old is None and u_new is not None:
            raise ValueError("advect_host: u_new without u_old")
        if u_old is not None:
            u_new = u_old if u_new is None else u_new
        checks = [("T_old", T_old, (self.n_nodes,))]
        if u_old is not None:
            checks += [("u_old", u_old, (self.n_nodes, self.dim)), ("u_new", u_new, (self.n_nodes, self.dim))]
        for name, t, shape in checks:
            if t.is_cuda or t.dtype != self.dtype or not t.is_contiguous() or not t.is_pinned():
                raise ValueError(f"{name} must be a contiguous, pinned {self.dtype} CPU tensor")
            if tuple(t.shape) != shape:
                raise ValueError(f"{name} must have shape {shape}")
        if out is None:
            out = torch.empty(self.n_nodes, dtype=self.dtype, pin_memory=True)
        elif out.is_cuda or out.dtype != self.dtype or not out.is_contiguous() or not out.is_pinned() \
                or tuple(out.shape) != (self.n_nodes,):
            raise ValueError(f"out must be a contiguous, pinned {self.dtype} CPU tensor of shape ({self.n_nodes},)")
        s = stream if stream is not None else torch.cuda.current_stream()
        up = (lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else None))  # noqa: E731
        check(_lib.load().elm_advect_host(self._h, up(u_old), up(u_new),
                                          ctypes.c_void_p(T_old.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                          float(dt), int(n_sub), ctypes.c_void_p(s.cuda_stream)))
        # the host tensors stay referenced until the stream has passed this call
        ev = torch.cuda.Event()
        ev.record(s)
        self._host_inflight = [x for x in self._host_inflight if not x[0].query()]
        self._host_inflight.append((ev, (T_old, u_old, u_new, out)))
        return out

    def advect_lookback(self, T_src: torch.Tensor, tau: float, b: int, n_sub: int = 1,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """Look-back distance b (Sec. 2.3.3) for a steady velocity: trace each
        node back b steps of ``tau`` (``n_sub`` RK4 substeps per step) and
        interpolate ``T_src`` = T^{n+1-b} there.  With T_src = T^0 and b = n+1
        this is the b = infinity scheme.  The trace over b steps is one call
        of ``advect`` with dt = b tau and b n_sub substeps."""
        if self._u is None:
            raise RuntimeError("set_velocity has not been called")
        if self._u[0] is not self._u[1]:
            raise ValueError("look-back over several steps needs a steady velocity")
        if b < 1:
            raise ValueError("b must be >= 1")
        return self.advect(T_src, b * tau, b * n_sub, out=out, stream=stream)

    def trace(self, D_in: torch.Tensor | None, dt: float, n_sub: int = 1, out: torch.Tensor | None = None,
              stream=None) -> torch.Tensor:
        """Continues the backward traces of every node over one interval of
        length dt with the current velocity pair (Sec. 2.3.3): starts at
        x_i + D_in[i] (at x_i when D_in is None) and returns the offsets
        X_i - x_i, [n_nodes, dim] in storage layout."""
        if D_in is not None:
            self._check_tensor(D_in, "D_in")
            if tuple(D_in.shape) != (self.n_nodes, self.dim):
                raise ValueError(f"D_in must have shape ({self.n_nodes}, {self.dim})")
        if out is None:
            out = torch.empty((self.n_nodes, self.dim), dtype=self.dtype, device=self.device)
        else:
            self._check_tensor(out, "out")
        check(_lib.load().elm_trace(self._h, ctypes.c_void_p(D_in.data_ptr()) if D_in is not None else None,
                                    ctypes.c_void_p(out.data_ptr()), float(dt), int(n_sub), _stream_ptr(stream)))
        return out

    def trace_eval(self, D: torch.Tensor, T_src: torch.Tensor, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
        """T_dst[i] = T_src_h(x_i + D[i]) at the end of traces from ``trace``."""
        self._check_tensor(D, "D")
        self._check_tensor(T_src, "T_src")
        if tuple(D.shape) != (self.n_nodes, self.dim) or T_src.shape != (self.n_nodes,):
            raise ValueError("D must be [n_nodes, dim] and T_src [n_nodes]")
        if out is None:
            out = torch.empty_like(T_src)
        else:
            self._check_tensor(out, "out")
        check(_lib.load().elm_trace_eval(self._h, ctypes.c_void_p(D.data_ptr()), ctypes.c_void_p(T_src.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
        return out

    def advect_lookback_unsteady(self, T_src: torch.Tensor, velocities, tau: float, n_sub: int = 1) -> torch.Tensor:
        """Look-back over a time-dependent velocity (Sec. 2.3.3): with
        ``velocities`` = [u^{n+1-b}, ..., u^{n+1}] (b + 1 nodal fields, storage
        layout) and T_src = T^{n+1-b}, traces every node back through the b
        intervals, newest first, each with its velocity pair, and interpolates
        T_src at the end (on the current stream).  Leaves the last pair
        (u^{n+1-b}, u^{n+2-b}) set as the mesh's velocity."""
        us = list(velocities)
        if len(us) < 2:
            raise ValueError("need at least two velocity fields (one interval)")
        bufs = [torch.empty((self.n_nodes, self.dim), dtype=self.dtype, device=self.device) for _ in range(2)]
        cur = None
        for j, k in enumerate(range(len(us) - 1, 0, -1)):
            if j == 0:
                self.set_velocity(us[k - 1], us[k])
            else:
                self.shift_velocity(us[k - 1])     # (u^{k-1}, u^k): u^k is the previous u_old
            cur = self.trace(cur, tau, n_sub, out=bufs[j % 2])
        return self.trace_eval(cur, T_src)

    def diffusion_step(self, c_hat: torch.Tensor, tau: float, kappa: float, theta: float = 1.0,
                       c_bnd: torch.Tensor | None = None, q: torch.Tensor | None = None, rtol: float | None = None,
                       max_iter: int = 1000, out: torch.Tensor | None = None, stream=None):
        """The diffusion solve of Eq. (linear system) (storage layout): returns
        (c_new, iterations, relative residual).  Needs ``diffusion=True`` at
        construction.  Synchronises the stream."""
        for name, t in (("c_hat", c_hat), ("c_bnd", c_bnd), ("q", q)):
            if t is not None:
                self._check_tensor(t, name)
                if t.shape != (self.n_nodes,):
                    raise ValueError(f"{name} must have shape ({self.n_nodes},)")
        if out is None:
            out = torch.empty_like(c_hat)
        else:
            self._check_tensor(out, "out")
        if rtol is None:
            rtol = 1e-11 if self.precision == "fp64" else 2e-6
        it = ctypes.c_int(0)
        res = ctypes.c_double(0.0)
        ptr = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
        check(_lib.load().elm_diffusion_step(self._h, ptr(c_hat), ptr(c_bnd), ptr(q), ptr(out), float(tau),
                                             float(kappa), float(theta), float(rtol), int(max_iter),
                                             ctypes.byref(it), ctypes.byref(res), _stream_ptr(stream)))
        return out, int(it.value), float(res.value)

    def strang_step(self, c: torch.Tensor, tau: float, kappa: float, n_sub: int = 1, theta: float = 1.0,
                    c_bnd: torch.Tensor | None = None, c_bnd_half: torch.Tensor | None = None, **solve):
        """One step of the Strang splitting (Algorithm 2): a diffusion solve
        over tau/2, the advection step over tau with the current velocity,
        and another diffusion solve over tau/2.  ``c_bnd_half`` / ``c_bnd``
        are the boundary values at t_n + tau/2 and t_{n+1} (None: keep c's)."""
        c1, _, _ = self.diffusion_step(c, 0.5 * tau, kappa, theta, c_bnd=c_bnd_half, **solve)
        c2 = self.advect(c1, tau, n_sub)
        c3, _, _ = self.diffusion_step(c2, 0.5 * tau, kappa, theta, c_bnd=c_bnd, **solve)
        return c3

    def advect_adjoint(self, T_old: torch.Tensor, gT_new: torch.Tensor, dt: float, n_sub: int = 1,
                       split: bool = True, stream=None):
        """Adjoint of ``advect`` for the current velocity: returns (gT_old,
        gU_old, gU_new) in storage layout; gU_new is None for a steady
        velocity or when ``split`` is False (then gU_old holds the sum).
        Needs ``adjoint=True`` at construction."""
        self._check_tensor(T_old, "T_old")
        self._check_tensor(gT_new, "gT_new")
        if self._u is None:
            raise RuntimeError("set_velocity has not been called")
        steady = self._u[0] is self._u[1]
        gT_old = torch.empty_like(T_old)
        gU_old = torch.empty((self.n_nodes, self.dim), dtype=self.dtype, device=T_old.device)
        gU_new = None if (steady or not split) else torch.empty_like(gU_old)
        check(_lib.load().elm_advect_adjoint(
            self._h, ctypes.c_void_p(T_old.data_ptr()), ctypes.c_void_p(gT_new.data_ptr()),
            ctypes.c_void_p(gT_old.data_ptr()), ctypes.c_void_p(gU_old.data_ptr()),
            ctypes.c_void_p(gU_new.data_ptr()) if gU_new is not None else None,
            float(dt), int(n_sub), _stream_ptr(stream)))
        return gT_old, gU_old, gU_new

    def status(self, stream=None) -> int:
        """Synchronises the stream and raises on a device-side condition."""
        check(_lib.load().elm_get_status(self._h, _stream_ptr(stream)))
        return _lib.ELM_OK


class Batch:
    """Many independent advection instances (meshes of one precision, any mix
    of dimensions and levels) advanced by one persistent kernel launch.

    Each mesh keeps its own velocity (``Mesh.set_velocity``).  ``advect`` takes
    lists of T_old / T_new tensors and per-instance dt and n_sub; it launches
    the batched kernel (one per element order) and the interface-copy pass on
    the current stream and can be captured in a CUDA graph.  ``blocks_per_sm``
    and ``chunks_per_item`` are the launch shape (see autotune.tune_batch).
    """

    def __init__(self, meshes, blocks_per_sm: int = 0, chunks_per_item: int = 1):
        lib = _lib.load()
        self.meshes = list(meshes)
        arr = (ctypes.c_void_p * len(self.meshes))(*[m.handle.value for m in self.meshes])
        h = ctypes.c_void_p()
        check(lib.elm_batch_create(arr, len(self.meshes), int(blocks_per_sm), int(chunks_per_item), ctypes.byref(h)))
        self._h = h
        self.blocks_per_sm = int(blocks_per_sm)
        self.chunks_per_item = int(chunks_per_item)
        self.n_items = int(lib.elm_batch_num_items(h))
        n = len(self.meshes)
        self._told = (ctypes.c_void_p * n)()
        self._tnew = (ctypes.c_void_p * n)()
        self._dt = (ctypes.c_double * n)()
        self._nsub = (ctypes.c_int * n)()

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _lib.load().elm_batch_destroy(h)
            self._h = None

    def advect(self, T_old, T_new, dt, n_sub, stream=None) -> None:
        n = len(self.meshes)
        if not (len(T_old) == len(T_new) == n):
            raise ValueError(f"expected {n} T_old / T_new tensors")
        dts = list(dt) if hasattr(dt, "__len__") else [float(dt)] * n
        subs = list(n_sub) if hasattr(n_sub, "__len__") else [int(n_sub)] * n
        for k, (m, a, b) in enumerate(zip(self.meshes, T_old, T_new)):
            m._check_tensor(a, "T_old")
            m._check_tensor(b, "T_new")
            if a.shape != (m.n_nodes,) or b.shape != (m.n_nodes,):
                raise ValueError(f"instance {k}: T must have shape ({m.n_nodes},)")
            self._told[k] = a.data_ptr()
            self._tnew[k] = b.data_ptr()
            self._dt[k] = float(dts[k])
            self._nsub[k] = int(subs[k])
        check(_lib.load().elm_batch_advect(self._h, self._told, self._tnew, self._dt, self._nsub,
                                           _stream_ptr(stream)))
