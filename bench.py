"""Benchmark of the MMOC advection step on GB300.

One step = one call of elm_advect over the whole mesh: every P2 node is
traced back with RK4 and T^n is interpolated at its departure point
(Algorithm 1 lines 3-4 of arXiv 2103.02388).  Prints ONE JSON line.

Default workload (the throughput target's configuration): unit cube, 6 Kuhn
macro tetrahedra, level 7 (257^3 = 16,974,593 P2 nodes), FP32, seeded
random-Fourier velocity (max |u| = 1), Gaussian cone, CFL 4, one RK4 substep.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload c3-l7-fp32|c2-l6-fp64|c3-l6-fp32]

N > 1 (under torchrun): every rank advects its own independent instance of the
workload (weak scaling, no data-path collective); the time is the maximum over
ranks and `value` counts the nodes of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (dim, level, precision, velocity, scalar, cfl, n_sub)
    "c3-l7-fp32": (3, 7, "fp32", "fourier", "gauss", 4.0, 1),
    "c3-l6-fp32": (3, 6, "fp32", "fourier", "gauss", 4.0, 1),
    "c2-l6-fp64": (3, 6, "fp64", "cellular", "slotted", 4.0, 1),
}
METRIC = "traced node updates/s per advection step (1 GPU), % of HBM roofline, err vs FP64 oracle"
# sources the advection kernel is compiled from: the DRAM traffic recorded in
# TRAFFIC_FILE is used only while their hash matches the one stored there
KERNEL_SRCS = [os.path.join(ROOT, "paper_2103_02388_gb300", "csrc", f)
               for f in ("advect.cu", "tracer.cuh", "elm_internal.h")]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "advect_traffic.json")


def _fields(spec, coords):
    from paper_2103_02388_gb300 import inputs
    dim, level, precision, vel, scal, cfl, n_sub = spec
    if vel == "fourier":
        u = inputs.random_fourier(coords, seed=3)
    else:
        u = inputs.cellular_flow(coords)
    if scal == "gauss":
        T = inputs.gaussian(coords, (0.35, 0.5, 0.5), 0.1)
    else:
        T = inputs.slotted_sphere(coords)
    if precision == "fp32":
        u = u.astype(np.float32).astype(np.float64)
        T = T.astype(np.float32).astype(np.float64)
    dt = inputs.dt_for_cfl(cfl, level, u)
    return u, T, dt


def _peaks():
    """(HBM GB/s, SM max MHz, kind) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


def alg_ops_per_node(dim: int, n_sub: int, steady: bool) -> int:
    """FP32/FP64 arithmetic operations the method needs per node and step
    (an FMA counts as one operation; index arithmetic is not counted).

    One P2 evaluation of the velocity at a stage point: stage point (dim FMA)
    and box clamp (2 dim), lattice coordinates (dim^2 FMA), floor and fraction
    (3 dim), macro barycentrics and their minimum (2 dim + 1), sort of the
    fractions (dim(dim-1)/2 compares), micro barycentrics (dim + 1), P2 basis
    (2 per node), sum (dim per node); the time interpolation doubles the sum
    and adds 2 dim.  The first stage of the first substep is the nodal value.
    RK4 combination per substep: 3 dim accumulations, dim update, 2 dim clamp.
    The final T evaluation: location as above (no stage point) plus basis and
    a 1-component sum.
    """
    nb = (dim + 1) * (dim + 2) // 2
    locate = dim * dim + 3 * dim + 2 * dim + 1 + dim * (dim - 1) // 2 + dim + 1
    vel = 3 * dim + locate + 2 * nb + dim * nb
    if not steady:
        vel += dim * nb + 2 * dim
    combine = 3 * dim + dim + 2 * dim
    t_eval = locate + 2 * nb + nb
    return (4 * n_sub - 1) * vel + n_sub * combine + t_eval


def alg_ops_split(dim: int, n_sub: int, steady: bool):
    """alg_ops_per_node split by the SM pipe each operation issues on: (FMA
    pipe: FMA, FADD, FMUL; ALU pipe: compares, min/max of the clamps and of the
    barycentric minimum, the floor of the cell index and the sort compares).
    The two parts add up to alg_ops_per_node."""
    nb = (dim + 1) * (dim + 2) // 2
    loc_fma = dim * dim + 2 * dim + 2 * (dim + 1)   # lattice coords, fraction and cell, both barycentrics
    loc_alu = 2 * dim + dim * (dim - 1) // 2        # floor, minimum, sort
    vel_fma = dim + loc_fma + 2 * nb + dim * nb + (0 if steady else dim * nb + 2 * dim)
    vel_alu = 2 * dim + loc_alu                     # stage-point clamp
    fma = (4 * n_sub - 1) * vel_fma + n_sub * 4 * dim + loc_fma + 3 * nb
    alu = (4 * n_sub - 1) * vel_alu + n_sub * 2 * dim + loc_alu
    assert fma + alu == alg_ops_per_node(dim, n_sub, steady)
    return fma, alu


def _device_props(index: int):
    """SM count, L2 size and name of the device, from its properties."""
    import torch
    p = torch.cuda.get_device_properties(index)
    return {"sms": int(p.multi_processor_count), "l2_bytes": getattr(p, "L2_cache_size", None), "name": p.name}


def _probe_pipes():
    """Pipe throughputs measured on this device by elm_probe_pipes (timed
    loops of FFMA, FFMA2, FP32 min/max, integer min/max and DFMA)."""
    import ctypes
    import torch
    from paper_2103_02388_gb300 import _lib
    r = (ctypes.c_double * 5)()
    _lib.check(_lib.load().elm_probe_pipes(r, 5, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)))
    return {"fp32_fma_per_s_ffma": r[0], "fp32_fma_per_s_ffma2": r[1], "fp32_minmax_per_s": r[2],
            "int32_minmax_per_s": r[3], "fp64_fma_per_s": r[4],
            "how": "elm_probe_pipes: 8 independent chains per thread, 8 x 256-thread blocks per SM, CUDA events"}


def _compute_roofline(precision, dim, n_sub, n_storage, alg_bytes, launch_ms, hbm_peak, sm_mhz, props, pipes,
                      util):
    """The compute side of the roofline, beside the HBM fraction: issue rate
    (warp instructions from the committed ncu record while the kernel's
    sources match it) and the algorithmic operations against the measured
    pipe peaks, with the time the algorithmic work alone would take at those
    peaks and the HBM fraction that time would allow."""
    t = launch_ms * 1e-3
    issue_peak = props["sms"] * 4 * sm_mhz * 1e6
    fma, alu = alg_ops_split(dim, n_sub, True)
    out = {"issue": {"peak": issue_peak, "unit": "warp instructions/s",
                     "peak_kind": f"unit counts: {props['sms']} SMs x 4 issue slots x {sm_mhz:.0f} MHz"}}
    if util is not None and util.get("warp_instructions"):
        wi = float(util["warp_instructions"])
        out["issue"].update({"achieved": wi / t, "frac": wi / t / issue_peak, "warp_instructions_per_launch": wi,
                             "source": "ncu smsp__inst_executed.sum of this kernel (profiles/advect_traffic.json)"})
    else:
        out["issue"].update({"achieved": None, "frac": None,
                             "source": "no ncu record for these kernel sources"})
    if precision == "fp32":
        fma_peak, alu_peak = pipes["fp32_fma_per_s_ffma2"], pipes["fp32_minmax_per_s"]
        ceil_s = max(fma * n_storage / fma_peak, alu * n_storage / alu_peak,
                     (fma / 2 + alu) * n_storage / 32 / issue_peak)
        out["fma_pipe"] = {"achieved": fma * n_storage / t, "peak": fma_peak, "unit": "FP32 FMA-pipe ops/s",
                           "frac": fma * n_storage / t / fma_peak, "ops_per_node": fma,
                           "peak_kind": "measured: FFMA2 loop, 2 FMAs per instruction"}
        out["alu_pipe"] = {"achieved": alu * n_storage / t, "peak": alu_peak, "unit": "ALU-pipe ops/s",
                           "frac": alu * n_storage / t / alu_peak, "ops_per_node": alu,
                           "peak_kind": "measured: FP32 min/max loop"}
        out["bound"] = "issue"
    else:
        ops = (fma + alu) * n_storage
        fp64_peak = pipes["fp64_fma_per_s"]
        ceil_s = ops / fp64_peak
        out["fp64_pipe"] = {"achieved": ops / t, "peak": fp64_peak, "unit": "FP64 ops/s", "frac": ops / t / fp64_peak,
                            "ops_per_node": fma + alu, "peak_kind": "measured: DFMA loop"}
        out["bound"] = "fp64 pipe"
    out["algorithmic_ceiling_ms"] = ceil_s * 1e3
    out["hbm_frac_at_ceiling"] = alg_bytes / ceil_s / 1e9 / hbm_peak
    return out


def _kernel_hash():
    h = hashlib.sha256()
    for p in KERNEL_SRCS:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _profile_record():
    """The committed ncu figures of the advection kernel, or None once the
    kernel's sources have changed since they were taken."""
    try:
        with open(TRAFFIC_FILE) as f:
            t = json.load(f)
        if t.get("kernel_sha") == _kernel_hash():
            return t
    except Exception:
        pass
    return None


def _traffic(workload):
    t = _profile_record()
    if t is not None and workload in t.get("per_launch_bytes", {}):
        return float(t["per_launch_bytes"][workload])
    return None


def _utilisation(workload):
    t = _profile_record()
    if t is not None and workload in t.get("utilisation", {}):
        return t["utilisation"][workload]
    return None


class ClockSampler:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            time.sleep(0.3)
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            self.proc.wait()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except (ValueError, IndexError):
                continue
            for name, val in zip(names, r[3:7]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(local_ms: float, local_units: int, dist=None, device=None):
    """Whole-job timing over ranks: the slowest rank's time and the units of
    all ranks (weak scaling, every rank advects its own instance)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return local_ms, local_units
    import torch
    t = torch.tensor([local_ms], dtype=torch.float64, device=device)
    n = torch.tensor([local_units], dtype=torch.int64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return float(t.item()), int(n.item())


def _oracle_mesh(spec):
    import oracle
    from paper_2103_02388_gb300 import inputs
    v, m = inputs.unit_cube() if spec[0] == 3 else inputs.unit_square()
    return oracle.OracleMesh(v, m, spec[1])


def _match_nodes(coords_ref, coords_other, M: int):
    """perm with coords_other[perm[i]] == coords_ref[i], for node sets on the
    1/M lattice of the unit square / cube (P2: M = 2^(L+1))."""
    def keys(c):
        q = np.rint(c * M).astype(np.int64)
        k = np.zeros(len(c), np.int64)
        for a in range(c.shape[1]):
            k = k * (M + 1) + q[:, a]
        return k
    ka, kb = keys(coords_ref), keys(coords_other)
    oa, ob = np.argsort(ka), np.argsort(kb)
    if not np.array_equal(ka[oa], kb[ob]):
        raise RuntimeError("node sets of the oracle and the library differ")
    perm = np.empty(len(ka), np.int64)
    perm[oa] = ob
    return perm


def _accuracy(spec, om, mesh, T0_storage, dt, steps: int = 3):
    """Error of the GPU step against the FP64 oracle on the same inputs (the
    FP32-rounded fields for an FP32 workload), over every unique node: after
    one step, and accumulated over ``steps`` steps with each side continuing
    from its own state.  Relative to max |T^0| (max) and ||T_oracle|| (L2)."""
    import torch
    u, T0, _ = _fields(spec, om.coords)
    n_sub = spec[6]
    perm = _match_nodes(om.coords, mesh.unique_coords(), mesh.order << mesh.level)
    Tg, out = T0_storage.clone(), torch.empty_like(T0_storage)
    To = T0
    tmax = float(np.abs(T0).max())
    res = {"reference": "FP64 oracle on the same inputs" + (" (FP32-rounded)" if spec[2] == "fp32" else ""),
           "nodes": int(om.n_nodes), "tolerance_one_step": 1e-5 if spec[2] == "fp32" else 1e-12}
    t0 = time.perf_counter()
    for k in range(1, steps + 1):
        mesh.advect(Tg, dt, n_sub, out=out)
        Tg, out = out, Tg
        To = om.advect(To, u, dt, n_sub)
        if k in (1, steps):
            g = mesh.to_unique(Tg).double().cpu().numpy()[perm]
            e = g - To
            rec = {"max_rel": float(np.abs(e).max() / tmax), "l2_rel": float(np.linalg.norm(e) / np.linalg.norm(To))}
            if k == 1:
                res["one_step"] = rec
            else:
                res["accumulated"] = dict(steps=steps, **rec)
    mesh.status()
    res["seconds"] = time.perf_counter() - t0
    return res


def _time_steps(mesh, T, dt, n_sub, steps, warmup, flush):
    """Mean CUDA-event time (ms) of ``steps`` elm_advect calls on the current
    stream, after ``warmup`` calls; L2 flushed between steps if asked."""
    import torch
    stream = torch.cuda.current_stream()
    a, b = T.clone(), torch.empty_like(T)
    scratch = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=T.device) if flush else None
    for _ in range(warmup):
        mesh.advect(a, dt, n_sub, out=b)
        a, b = b, a
    torch.cuda.synchronize()
    ev = []
    for i in range(steps):
        if flush:
            scratch.fill_(float(i))
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        mesh.advect(a, dt, n_sub, out=b)
        e.record(stream)
        ev.append((s, e))
        a, b = b, a
    torch.cuda.synchronize()
    mesh.status()
    return float(np.mean([s.elapsed_time(e) for s, e in ev]))


def _fp64_record(dev, hbm_peak, sm_mhz, props, pipes, with_oracle: bool, steps: int = 20, warmup: int = 3):
    """Config 2's plain FP64 step on the GPU (unit cube, level 6, cellular
    flow, slotted sphere, CFL 4): time per step, throughput, the FP64-pipe and
    HBM fractions, and (with the oracle) its error against the FP64 oracle."""
    import torch
    from paper_2103_02388_gb300 import elm, inputs
    spec = WORKLOADS["c2-l6-fp64"]
    dim, level, _, vel, scal, cfl, n_sub = spec
    mesh = elm.Mesh(*inputs.unit_cube(), level, "fp64")
    u, T0, dt = _fields(spec, mesh.unique_coords())
    mesh.set_velocity(mesh.to_storage(torch.tensor(u, dtype=torch.float64, device=dev)))
    T = mesh.to_storage(torch.tensor(T0, dtype=torch.float64, device=dev))
    alg_bytes = mesh.n_nodes * (dim * 8 + 16)
    ms = _time_steps(mesh, T, dt, n_sub, steps, warmup, flush=alg_bytes < 2 * (props["l2_bytes"] or 129 * 2**20))
    rec = {"workload": "c2-l6-fp64", "level": level, "unique_nodes": mesh.n_unique, "velocity": vel, "scalar": scal,
           "cfl": cfl, "n_sub": n_sub, "steps": steps, "ms_per_step": ms,
           "value": mesh.n_unique / (ms * 1e-3), "unit": "node updates/s",
           "l2": "flushed between steps (256 MB write)",
           "hbm": {"achieved": alg_bytes / (ms * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
                   "frac": alg_bytes / (ms * 1e-3) / 1e9 / hbm_peak, "algorithmic_bytes_per_launch": alg_bytes},
           "compute": _compute_roofline("fp64", dim, n_sub, mesh.n_nodes, alg_bytes, ms, hbm_peak, sm_mhz, props,
                                        pipes, _utilisation("c2-l6-fp64"))}
    if with_oracle:
        rec["accuracy"] = _accuracy(spec, _oracle_mesh(spec), mesh, T, dt)
    return rec


def _accumulated_record(dev, steps: int = 100, checkpoints=(1, 10, 25, 50, 100)):
    """Config 3's error budget over a 100-step rollout at level 6 (random
    Fourier velocity, Gaussian cone, CFL 4): the FP32 GPU path and the plain
    FP64 GPU path, both on the FP32-rounded inputs, against the FP64 oracle
    and against each other, accumulated (each side continuing from its own
    state) and per step (one step of each GPU path from the oracle's state
    against the oracle's step).  Relative to max |T^0| (max) and to the
    reference's norm (L2)."""
    import torch
    from paper_2103_02388_gb300 import elm, inputs
    spec = WORKLOADS["c3-l6-fp32"]
    dim, level, _, _, _, cfl, n_sub = spec
    om = _oracle_mesh(spec)
    u, T0, dt = _fields(spec, om.coords)          # FP32-rounded fields, in FP64
    g32 = elm.Mesh(*inputs.unit_cube(), level, "fp32")
    g64 = elm.Mesh(*inputs.unit_cube(), level, "fp64")
    perm = _match_nodes(om.coords, g32.unique_coords(), g32.order << level)
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))

    def to_dev(mesh, a, dtype):
        return mesh.to_storage(torch.tensor(a[inv], dtype=dtype, device=dev))

    def to_host(mesh, t):
        return mesh.to_unique(t).double().cpu().numpy()[perm]
    g32.set_velocity(to_dev(g32, u, torch.float32))
    g64.set_velocity(to_dev(g64, u, torch.float64))
    tmax = float(np.abs(T0).max())

    def err(a, ref):
        e = a - ref
        return {"max_rel": float(np.abs(e).max() / tmax), "l2_rel": float(np.linalg.norm(e) / np.linalg.norm(ref))}
    T32, T64, To = to_dev(g32, T0, torch.float32), to_dev(g64, T0, torch.float64), T0.copy()
    rows = []
    t0 = time.perf_counter()
    for k in range(1, steps + 1):
        prev = To
        T32, T64 = g32.advect(T32, dt, n_sub), g64.advect(T64, dt, n_sub)
        To = om.advect(To, u, dt, n_sub)
        if k in checkpoints:
            h32, h64 = to_host(g32, T32), to_host(g64, T64)
            one32 = to_host(g32, g32.advect(to_dev(g32, prev, torch.float32), dt, n_sub))
            one64 = to_host(g64, g64.advect(to_dev(g64, prev, torch.float64), dt, n_sub))
            rows.append({"step": k,
                         "accumulated": {"fp32_vs_oracle": err(h32, To), "fp32_vs_fp64_gpu": err(h32, h64),
                                         "fp64_gpu_vs_oracle": err(h64, To)},
                         "per_step": {"fp32_vs_oracle": err(one32, To), "fp64_gpu_vs_oracle": err(one64, To)}})
    g32.status()
    g64.status()
    return {"workload": "c3-l6-fp32 (config 3 at level 6)", "level": level, "unique_nodes": int(om.n_nodes),
            "cfl": cfl, "n_sub": n_sub, "dt": dt, "steps": steps,
            "inputs": "FP32-rounded velocity and T^0 for every side", "tolerance_per_step": {"fp32": 1e-5, "fp64": 1e-12},
            "rows": rows, "seconds": time.perf_counter() - t0}


def _cpu_baseline(spec, seconds: float = 12.0, om=None):
    """The CPU oracle timed on a bounded sample of the same workload."""
    import oracle
    om = _oracle_mesh(spec) if om is None else om
    u, T, dt = _fields(spec, om.coords)
    threads = oracle.default_threads()
    rng = np.random.default_rng(1)
    n = 20000
    while True:
        idx = np.sort(rng.choice(om.n_nodes, min(n, om.n_nodes), replace=False))
        t0 = time.perf_counter()
        om.advect_nodes(T, u, dt, idx, n_sub=spec[6], threads=threads)
        el = time.perf_counter() - t0
        if el >= seconds / 4 or len(idx) == om.n_nodes:
            break
        n = int(n * min(8.0, max(2.0, seconds / 2 / max(el, 1e-3))))
    # the same oracle on one thread, on a sample sized for about the same time
    n1 = max(1000, min(len(idx), int(len(idx) / max(threads, 1))))
    idx1 = np.sort(rng.choice(om.n_nodes, n1, replace=False))
    t0 = time.perf_counter()
    om.advect_nodes(T, u, dt, idx1, n_sub=spec[6], threads=1)
    el1 = time.perf_counter() - t0
    return {"value": len(idx) / el, "unit": "node updates/s", "cores": threads, "kind": "oracle",
            "sample": (f"all {len(idx)} nodes of the workload" if len(idx) == om.n_nodes else
                       f"{len(idx)} random nodes of the same workload") + f", one step, FP64, {threads} threads",
            "seconds": el, "cpu_model": _cpu_model(),
            "single_thread": {"value": n1 / el1, "unit": "node updates/s", "sample": f"{n1} random nodes, one step",
                              "seconds": el1}}


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:  # Arm hosts: /proc/cpuinfo has no model name, lscpu names the core
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def run_reference(args, spec):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    import oracle
    from paper_2103_02388_gb300 import inputs
    dim, level = spec[0], spec[1]
    v, m = inputs.unit_cube() if dim == 3 else inputs.unit_square()
    om = oracle.OracleMesh(v, m, level)
    u, T, dt = _fields(spec, om.coords)
    threads = oracle.default_threads()
    n = min(om.n_nodes, 60000)
    rng = np.random.default_rng(2)
    idx = np.sort(rng.choice(om.n_nodes, n, replace=False))
    for _ in range(warm):
        om.advect_nodes(T, u, dt, idx[: n // 10], n_sub=spec[6], threads=threads)
    t0 = time.perf_counter()
    for _ in range(steps):
        om.advect_nodes(T, u, dt, idx, n_sub=spec[6], threads=threads)
    el = time.perf_counter() - t0
    val = n * steps / el
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "node updates/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "sample_nodes": n},
        "cpu_baseline": {"kind": "oracle", "cores": threads, "value": val, "unit": "node updates/s",
                         "sample": f"{n} random nodes per step of the {args.workload} workload"},
        "e2e": {"value": val, "unit": "node updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_ours(args, spec):
    import torch
    from paper_2103_02388_gb300 import elm, inputs

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dim, level, precision, vel, scal, cfl, n_sub = spec
    v, m = inputs.unit_cube() if dim == 3 else inputs.unit_square()
    mesh = elm.Mesh(v, m, level, precision, host_staging=True)
    ucoords = mesh.unique_coords()
    u, T0, dt = _fields(spec, ucoords)
    dtype = mesh.dtype
    u_s = mesh.to_storage(torch.tensor(u, dtype=dtype, device=dev))
    T_a = mesh.to_storage(torch.tensor(T0, dtype=dtype, device=dev))
    T_init = T_a.clone()
    T_b = torch.empty_like(T_a)
    mesh.set_velocity(u_s)
    stream = torch.cuda.current_stream()
    n_storage, n_unique = mesh.n_nodes, mesh.n_unique
    esz = 8 if precision == "fp64" else 4
    alg_bytes = n_storage * (dim * esz + 2 * esz)     # read u + read T_old + write T_new
    working_set = alg_bytes
    props = _device_props(local)
    l2_bytes = props["l2_bytes"] or 129 * 2**20
    flush = working_set < 2 * l2_bytes
    scratch = torch.empty(256 * 2**20 // 4, dtype=torch.float32, device=dev) if flush else None

    def step(src, dst):
        mesh.advect(src, dt, n_sub, out=dst)

    for _ in range(args.warmup):
        step(T_a, T_b)
        T_a, T_b = T_b, T_a
    torch.cuda.synchronize()
    mesh.status()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clocks:
        for i in range(args.steps):
            if flush:
                scratch.fill_(float(i))
            starts[i].record(stream)
            step(T_a, T_b)
            ends[i].record(stream)
            T_a, T_b = T_b, T_a
        torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    mesh.status()
    times = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms, units = aggregate(float(sum(times)), n_unique * args.steps, dist, dev)
    ms_per_step = total_ms / args.steps
    value = units / (total_ms * 1e-3)

    # end to end through the public API with host buffers (elm_advect_host):
    # every step copies its inputs (u and T_old) from pinned host memory to
    # the device and its result T_new back; consecutive steps overlap their
    # copies with the previous step's kernel on the mesh's copy streams
    u_h = u_s.cpu().pin_memory()
    T_h = T_a.cpu().pin_memory()
    out_h = torch.empty_like(T_h).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    for _ in range(3):
        mesh.advect_host(T_h, dt, n_sub, u_old=u_h, out=out_h)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mesh.advect_host(T_h, dt, n_sub, u_old=u_h, out=out_h)
    torch.cuda.synchronize()
    e2e_ms, e2e_units = aggregate((time.perf_counter() - t0) * 1e3, n_unique * e2e_steps, dist, dev)
    mesh.status()
    # the host path computes what the device path computes, bit for bit
    mesh.set_velocity(u_s)
    if not torch.equal(out_h, mesh.advect(T_h.to(dev), dt, n_sub).cpu()):
        raise RuntimeError("host-buffer step differs from the device step")
    e2e = {"value": e2e_units / (e2e_ms * 1e-3), "unit": "node updates/s",
           "h2d_bytes_per_step": int(u_h.numel() * esz + T_h.numel() * esz),
           "d2h_bytes_per_step": int(out_h.numel() * esz),
           "path": "elm_advect_host: pinned host buffers, copies pipelined with the previous step"}
    # the same with the (steady) velocity resident on the device: the
    # velocity is given once, then each step moves T^n in and T^{n+1} out
    mesh.advect_host(T_h, dt, n_sub, u_old=u_h, out=out_h)
    for _ in range(3):
        mesh.advect_host(T_h, dt, n_sub, out=out_h)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        mesh.advect_host(T_h, dt, n_sub, out=out_h)
    torch.cuda.synchronize()
    res_ms, res_units = aggregate((time.perf_counter() - t0) * 1e3, n_unique * e2e_steps, dist, dev)
    mesh.status()
    e2e_resident = {"value": res_units / (res_ms * 1e-3), "unit": "node updates/s",
                    "h2d_bytes_per_step": int(T_h.numel() * esz), "d2h_bytes_per_step": int(out_h.numel() * esz),
                    "path": "elm_advect_host with the velocity resident (given once): T^n in, T^{n+1} out"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    hbm_peak, sm_mhz, peak_kind = _peaks()
    hbm_achieved = alg_bytes / (ms_per_step * 1e-3) / 1e9
    pipes = _probe_pipes()
    compute = _compute_roofline(precision, dim, n_sub, n_storage, alg_bytes, ms_per_step, hbm_peak, sm_mhz, props,
                                pipes, _utilisation(args.workload))
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "node updates/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {
            "workload": args.workload,
            "mesh": f"unit {'cube, 6 Kuhn macro tetrahedra' if dim == 3 else 'square, 2 macro triangles'}",
            "level": level, "unique_nodes": n_unique, "storage_nodes": n_storage, "velocity": vel,
            "scalar": scal, "cfl": cfl, "n_sub": n_sub, "dt": dt,
            "l2": "flushed between steps (256 MB write)" if flush else "inputs larger than L2 (not flushed)",
            "parallelism": f"{world} independent replicas" if world > 1 else "1 GPU",
            "device": props,
        },
        # the metric's roofline: algorithmic bytes of a step (read u, read T^n,
        # write T^{n+1}) over the CUDA-event time of the step, against the
        # measured HBM copy bandwidth; the compute side sits beside it
        "roofline": {"bound": "hbm", "achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": hbm_achieved / hbm_peak,
                     "peak_kind": ("measured (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured"
                                   else "fallback: 6.8 TB/s, the profiling recipe's figure"),
                     "traffic": _traffic(args.workload), "algorithmic_bytes_per_launch": alg_bytes,
                     "kernel": "k_advect (+ k_ghost_copy, about 1% of the step)", "avg_launch_ms": ms_per_step,
                     "compute": compute, "pipes": pipes,
                     "ncu_utilisation": _utilisation(args.workload)},
        # per step: k_advect, then k_ghost_copy for the interface copies
        "gpu_launches": args.steps * (2 if n_storage > n_unique else 1),
        "clocks": clocks.summary(),
        "e2e": e2e,
        "e2e_resident_velocity": e2e_resident,
    }
    if world == 1:
        # the plain FP64 form of the step (config 2), timed the same way
        line["fp64"] = _fp64_record(dev, hbm_peak, sm_mhz, props, pipes, with_oracle=not args.no_cpu_baseline)
    if world == 1 and not args.no_cpu_baseline:
        om = _oracle_mesh(spec)
        line["accuracy"] = _accuracy(spec, om, mesh, T_init, dt)
        line["cpu_baseline"] = _cpu_baseline(spec, om=om)
        del om
        line["accumulated_100"] = _accumulated_record(dev)
        line["other_forms"] = _other_forms()
    print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def _other_forms():
    """The batched form (config 4, FP32), the differentiated rollout (config
    5, FP32) and the diffusion solve (level 6, FP64) measured in the default
    run, each as its own workload would report it (compact)."""
    import argparse as _ap
    out = {}

    def keep(rec, keys):
        return {k: rec[k] for k in keys if k in rec}
    try:
        r = run_batch(_ap.Namespace(workload="c4-batch-fp32", steps=100, warmup=3), emit=False)
        out["c4-batch-fp32"] = keep(r, ("metric", "value", "unit", "ms_per_step", "steps", "gpu_launches")) | {
            "autotune": {k: r["config"]["autotune"][k] for k in ("blocks_per_sm", "chunks_per_item")},
            "graph": r["config"]["graph"], "instances": r["config"]["instances"],
            "hbm_frac": r["roofline"]["frac"]}
        r = run_adjoint(_ap.Namespace(workload="c5-adjoint-l6-fp32", steps=50, warmup=1), emit=False)
        out["c5-adjoint-l6-fp32"] = keep(r, ("metric", "value", "unit", "ms_per_step", "steps")) | {
            "timed": r["config"]["timed"]}
        r = run_diffusion(_ap.Namespace(workload="diffusion-l6-fp64", steps=10, warmup=2), emit=False)
        out["diffusion-l6-fp64"] = keep(r, ("metric", "value", "unit", "ms_per_solve", "cg_iterations",
                                            "relative_residual")) | {"solver": r["config"]["solver"],
                                                                     "hbm_frac": r["roofline"]["frac"]}
    except Exception as e:  # reported, never hides the main record
        out["error"] = f"{type(e).__name__}: {e}"
    return out


DIFFUSION_WORKLOADS = {
    # name: (dim, level, precision, order, tau, kappa, theta)
    "diffusion-l6-fp64": (3, 6, "fp64", 2, 0.01, 0.01, 1.0),
    "diffusion-l6-fp32": (3, 6, "fp32", 2, 0.01, 0.01, 1.0),
}


def run_diffusion(args, emit: bool = True):
    """The diffusion solve of Eq. (linear system) on the unit cube (P2, 6 Kuhn
    macros): CUDA-event time of whole elm_diffusion_step calls, CG iterations,
    and the compulsory bytes of one CG iteration (operator apply plus vector
    updates, storage layout) against the measured HBM peak."""
    import torch
    from paper_2103_02388_gb300 import elm, inputs
    dim, level, precision, order, tau, kappa, theta = DIFFUSION_WORKLOADS[args.workload]
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, level, precision, order=order, diffusion=True)
    x = mesh.unique_coords()
    c0 = inputs.gaussian(x, (0.35, 0.5, 0.5), 0.1) + 0.2 * x[:, 0]
    c = mesh.to_storage(torch.tensor(c0, dtype=mesh.dtype, device="cuda"))
    out = torch.empty_like(c)
    for _ in range(args.warmup):
        mesh.diffusion_step(c, tau, kappa, theta, out=out)
    torch.cuda.synchronize()
    times, iters = [], []
    with ClockSampler(0) as clocks:
        for _ in range(args.steps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record()
            _, it, res = mesh.diffusion_step(c, tau, kappa, theta, out=out)
            e.record()
            torch.cuda.synchronize()
            times.append(s.elapsed_time(e))
            iters.append(it)
    # FP64 meshes solve by defect correction: the iterations counted are the
    # FP32 PCG iterations of the corrections (their vectors are FP32), plus a
    # few FP64 residuals
    esz = 4
    n, ns = mesh.n_unique, mesh.n_nodes
    # per CG iteration, vectors in the storage layout (ns slots): operator (read
    # p, write q), update (x, r read + write; p, q, inverse diagonal read; z
    # write; the 1-byte dot-product mask), direction (read z, p; write p).  The
    # operator's own tables (interior node lists, face rows) are not counted.
    bytes_iter = ns * (esz * (2 + 8 + 3) + 1)
    ms = float(np.median(times))
    it = int(np.median(iters))
    ms_iter = ms / max(it, 1)
    hbm_peak, _, kind = _peaks()
    achieved = bytes_iter / (ms_iter * 1e-3) / 1e9
    rec = {
        "metric": "diffusion solve (Eq. linear system): unknown updates per second (CG iterations x unknowns / s)",
        "value": n * it / (ms * 1e-3), "unit": "unknown updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_solve": ms, "cg_iterations": it, "ms_per_iteration": ms_iter,
        "relative_residual": res, "higher_is_better": True, "dtype": "f64" if precision == "fp64" else "f32",
        "data": "synthetic",
        "config": {"workload": args.workload, "mesh": "unit cube, 6 Kuhn macro tetrahedra", "level": level,
                   "order": order, "unique_nodes": n, "tau": tau, "kappa": kappa, "theta": theta,
                   "solver": ("defect correction: FP64 residuals, FP32 Jacobi-PCG corrections" if precision == "fp64"
                              else "FP32 Jacobi-PCG")},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": kind, "bytes_per_iteration": bytes_iter,
                     "scope": "one FP32 CG iteration (all its kernels), averaged over the solve"},
        "clocks": clocks.summary()}
    if emit:
        print(json.dumps(rec))
    return rec


VARIANT_WORKLOADS = {
    # P1 elements (Sec. 3.1): the same node count as the default P2 workload
    # (257^3 unique nodes at level 8), one advection step per launch
    "c3-l8-p1-fp32": {"dim": 3, "level": 8, "precision": "fp32", "order": 1, "cfl": 4.0, "mode": "step"},
    # look-back over the time-dependent swirling flow (Sec. 3.3, Table 3's
    # 129^3-node P1 mesh, tau = 0.025): one interval of elm_trace per step,
    # with the interval's older velocity packed by elm_shift_velocity (the
    # newer one is the previous interval's older one)
    "swirl-l7-p1-fp32-trace": {"dim": 3, "level": 7, "precision": "fp32", "order": 1, "tau": 0.025,
                               "mode": "trace"},
    # the blended annulus (Sec. 3.4 geometry: 6 sectors x 2 layers, P2, FP64),
    # rotation about the origin, tau = 2 pi / 63 as in Table 4
    "annulus-l8-fp64": {"dim": 2, "level": 8, "precision": "fp64", "order": 2, "mode": "annulus"},
}


def run_variant(args):
    """P1 and trace forms of the advection kernel: CUDA-event time per step
    on the launching stream, with the HBM roofline of their compulsory bytes."""
    import torch
    from paper_2103_02388_gb300 import elm, inputs
    w = VARIANT_WORKLOADS[args.workload]
    dim, level, precision = w["dim"], w["level"], w["precision"]
    if w["mode"] == "annulus":
        v, m = inputs.annulus_ring(6, 2)
        mesh = elm.Mesh(v, m, level, precision, order=w["order"], annulus=(0.5, 1.5, 6, 0.0))
    else:
        v, m = inputs.unit_cube()
        mesh = elm.Mesh(v, m, level, precision, order=w["order"])
    x = mesh.unique_coords()
    esz = 8 if precision == "fp64" else 4
    n, ns = mesh.n_unique, mesh.n_nodes
    stream = torch.cuda.current_stream()
    tg = lambda a: mesh.to_storage(torch.tensor(a, dtype=mesh.dtype, device="cuda"))  # noqa: E731
    if w["mode"] in ("step", "annulus"):
        if w["mode"] == "step":
            u = inputs.random_fourier(x, seed=3)
            dt = inputs.dt_for_cfl(w["cfl"], level, u)
            T0 = inputs.gaussian(x, (0.35, 0.5, 0.5), 0.1)
        else:
            u = np.stack([-x[:, 1], x[:, 0]], axis=1)
            dt = 2 * np.pi / 63
            T0 = inputs.heat_kernel_rotating(x, 2 * np.pi * 1e-3 / 1e-7, 1e-7)
        mesh.set_velocity(tg(u))
        Ta = tg(T0)
        Tb = torch.empty_like(Ta)

        def step(i):
            nonlocal Ta, Tb
            mesh.advect(Ta, dt, 1, out=Tb)
            Ta, Tb = Tb, Ta
        alg_bytes = ns * (dim * esz + 2 * esz)
        launches = 1
        cfg = {"cfl": w.get("cfl"), "dt": dt}
    else:
        tau = w["tau"]
        K = int(round(1.5 / tau))
        fields = [tg(inputs.swirl_3d(x, k * tau)) for k in range(K + 1)]
        D = [torch.zeros((ns, dim), dtype=mesh.dtype, device="cuda") for _ in range(2)]

        def step(i):
            k = K - (i % K)
            if i % K == 0:
                mesh.set_velocity(fields[k - 1], fields[k])
            else:
                mesh.shift_velocity(fields[k - 1])   # u^k is the previous interval's u_old
            mesh.trace(D[i % 2] if i % K else None, tau, 1, out=D[(i + 1) % 2])
        # read u^{k-1}, u^k ([n, 3] each), read D_in, write D_out
        alg_bytes = ns * (2 * dim * esz + 2 * dim * esz)
        launches = 3
        cfg = {"tau": tau, "intervals": K}
    for i in range(args.warmup):
        step(i)
    torch.cuda.synchronize()
    mesh.status()
    times = []
    with ClockSampler(0) as clocks:
        for i in range(args.steps):
            s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s.record(stream)
            step(args.warmup + i)
            e.record(stream)
            times.append((s, e))
        torch.cuda.synchronize()
    mesh.status()
    ms = float(np.mean([s.elapsed_time(e) for s, e in times]))
    hbm_peak, _, kind = _peaks()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    print(json.dumps({
        "metric": "traced node updates/s per look-back interval (1 GPU)" if w["mode"] == "trace" else
                  "traced node updates/s per step (1 GPU)",
        "value": n / (ms * 1e-3), "unit": "node updates/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f64", "data": "synthetic",
        "config": dict({"workload": args.workload,
                        "mesh": ("annulus 0.5 <= |x| <= 1.5, 6 x 2 ring blended (polar map)" if w["mode"] == "annulus"
                                 else "unit cube, 6 Kuhn macro tetrahedra"), "level": level,
                        "order": w["order"], "unique_nodes": n, "storage_nodes": ns,
                        "l2": "inputs larger than L2 (not flushed)"}, **cfg),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": kind, "algorithmic_bytes_per_step": alg_bytes,
                     "kernel": {"step": "k_advect (P1)", "trace": "k_advect (kTrace) + k_pack_velocity (one field) + k_ghost_copy",
                                "annulus": "k_advect (blended)"}[w["mode"]]},
        "gpu_launches": launches * args.steps, "clocks": clocks.summary()}))


BATCH_WORKLOADS = {
    # 64 independent instances (2D levels 4-8, 3D levels 4-6), one CUDA graph of the time loop
    "c4-batch-fp32": "fp32",
    "c4-batch-fp64": "fp64",
}


def run_batch(args, emit: bool = True):
    """The batched form: every instance of the seeded recipe advanced by one
    persistent launch per step, the time loop of ``steps`` steps captured in
    one CUDA graph; launch shape from the autotuner.  Time = CUDA events
    around one replay of the graph on its stream."""
    import torch
    from paper_2103_02388_gb300 import elm, inputs
    from paper_2103_02388_gb300.autotune import tune_batch
    precision = BATCH_WORKLOADS[args.workload]
    recipe = inputs.batch_recipe(seed=4, count=64)
    meshes, Ta, Tb, dts, subs = [], [], [], [], []
    nodes = storage = alg_bytes = 0
    esz = 8 if precision == "fp64" else 4
    for e in recipe:
        v, m = inputs.unit_cube() if e["dim"] == 3 else inputs.unit_square()
        gm = elm.Mesh(v, m, e["level"], precision)
        u, T, dt = inputs.batch_fields(e, gm.node_coords())
        gm.set_velocity(torch.tensor(u, dtype=gm.dtype, device="cuda"))
        meshes.append(gm)
        Ta.append(torch.tensor(T, dtype=gm.dtype, device="cuda"))
        Tb.append(torch.empty_like(Ta[-1]))
        dts.append(dt)
        subs.append(1)
        nodes += gm.n_unique
        storage += gm.n_nodes
        alg_bytes += gm.n_nodes * (e["dim"] * esz + 2 * esz)
    tune = tune_batch(meshes, Ta, Tb, dts, subs, reps=3)
    batch = elm.Batch(meshes, tune["blocks_per_sm"], tune["chunks_per_item"])
    stream = torch.cuda.Stream()
    stream.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            batch.advect(Ta, Tb, dts, subs)
            Ta, Tb = Tb, Ta
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        x, y = Ta, Tb
        for _ in range(args.steps):
            batch.advect(x, y, dts, subs)
            x, y = y, x
    graph.replay()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        with torch.cuda.stream(stream):
            ev0.record(stream)
            graph.replay()
            ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    for gm in meshes:
        gm.status()
    hbm_peak, _, kind = _peaks()
    achieved = alg_bytes / (ms * 1e-3) / 1e9
    rec = {
        "metric": "traced node updates/s per batched step (1 GPU)", "value": nodes / (ms * 1e-3),
        "unit": "node updates/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(meshes), "unique_nodes": nodes,
                   "storage_nodes": storage, "recipe": "inputs.batch_recipe(seed=4, count=64)",
                   "graph": f"{args.steps} steps in one CUDA graph", "autotune": tune,
                   "l2": "inputs larger than L2 (not flushed)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "peak_kind": kind, "algorithmic_bytes_per_step": alg_bytes,
                     "kernel": "k_advect_batch"},
        # per step: the batched kernel (one per element order present) and the
        # interface-copy pass
        "gpu_launches": args.steps * (len({m.order for m in meshes}) + 1), "clocks": clocks.summary()}
    if emit:
        print(json.dumps(rec))
    return rec


ADJOINT_WORKLOADS = {
    # 3D level 6, cellular flow, 50 steps, checkpoints every 10, loss 0.5 ||T^50 - T*||^2
    "c5-adjoint-l6-fp64": "fp64",
    "c5-adjoint-l6-fp32": "fp32",
}


def run_adjoint(args, emit: bool = True):
    """Gradient of a 50-step rollout (Sec. 2.3.1 step, differentiated): the
    forward steps, the recomputation inside checkpointed segments and the
    adjoint steps, for T^0 and the velocity.  One 'step' of the metric is one
    forward step plus its share of the backward pass."""
    import torch
    from paper_2103_02388_gb300 import autograd, elm, inputs
    precision = ADJOINT_WORKLOADS[args.workload]
    level, steps_roll, every = 6, 50, 10
    v, m = inputs.unit_cube()
    mesh = elm.Mesh(v, m, level, precision, adjoint=True)
    x = mesh.unique_coords()
    tg = lambda a: mesh.to_storage(torch.tensor(a, dtype=mesh.dtype, device="cuda"))  # noqa: E731
    u = inputs.cellular_flow(x)
    dt = inputs.dt_for_cfl(4.0, level, u)
    T0 = tg(inputs.gaussian(x, (0.35, 0.5, 0.5), 0.1))
    Tstar = tg(inputs.random_fourier(x, seed=5)[:, 0])
    u_s = tg(u)

    def one():
        T = T0.clone().requires_grad_(True)
        uu = u_s.clone().requires_grad_(True)
        loss = 0.5 * ((autograd.rollout(T, uu, mesh, dt, steps_roll, 1, every) - Tstar) ** 2).sum()
        loss.backward()
        return T.grad, uu.grad
    for _ in range(max(1, args.warmup)):
        one()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    reps = max(1, args.steps // steps_roll)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clocks:
        ev0.record(stream)
        for _ in range(reps):
            gT, gU = one()
        ev1.record(stream)
        torch.cuda.synchronize()
    mesh.status()
    if not (torch.isfinite(gT).all() and torch.isfinite(gU).all()):
        raise RuntimeError("non-finite gradient")
    ms = ev0.elapsed_time(ev1) / (reps * steps_roll)
    rec = {
        "metric": "node updates/s of forward + adjoint per step of a checkpointed rollout (1 GPU)",
        "value": mesh.n_unique / (ms * 1e-3), "unit": "node updates/s", "n_gpus": 1,
        "steps": reps * steps_roll, "warmup": max(1, args.warmup), "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if precision == "fp32" else "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "mesh": "unit cube, 6 Kuhn macro tetrahedra", "level": level,
                   "unique_nodes": mesh.n_unique, "velocity": "cellular", "cfl": 4.0, "rollout_steps": steps_roll,
                   "checkpoint_every": every, "loss": "0.5 ||T^50 - T*||^2, T* = random Fourier (seed 5)",
                   "timed": f"{reps} gradient(s) of the whole rollout, CUDA events (host launch gaps included)"},
        "gpu_launches": None, "clocks": clocks.summary()}
    if emit:
        print(json.dumps(rec))
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c3-l7-fp32",
                    choices=sorted(WORKLOADS) + sorted(DIFFUSION_WORKLOADS) + sorted(VARIANT_WORKLOADS)
                    + sorted(BATCH_WORKLOADS) + sorted(ADJOINT_WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.workload in DIFFUSION_WORKLOADS:
        run_diffusion(args)
        return
    if args.workload in VARIANT_WORKLOADS:
        run_variant(args)
        return
    if args.workload in BATCH_WORKLOADS:
        run_batch(args)
        return
    if args.workload in ADJOINT_WORKLOADS:
        run_adjoint(args)
        return
    spec = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, spec)
    else:
        run_ours(args, spec)


if __name__ == "__main__":
    main()
