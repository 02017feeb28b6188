"""Throughput benchmark: GDOF-stage/s of the hybrid-mesh DG right-hand side + time-step update.

Workload: the 64x64x80-cell layered hybrid mesh on [-1,1]^3 (layers
H x34 | W x2 | H x36 | T | K x4 | U | H x2: 294,912 hex, 16,384 wedges, 40,960
pyramids, 114,688 tets), order N = 4 (44,359,680 DOFs x 4 fields), wave speed
1.0 / 1.5 alternating by layer, upwind flux, two time-step levels.

Headline: one step = one coarse step of the two-level multi-rate AB3 scheme
(every element's rhs once, the fine level's rhs a second time, AB3 updates);
GDOF-stage/s = (ndof + ndof_fine) * steps / time, i.e. the element-stages
actually performed.  Beside it ("single_rate"): one step = one LSRK(5,4) step
(five fused stage kernels per element type), GDOF-stage/s = ndof * 5 * steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

Beside them ("sem_hex"): the multi-rate workload with SEM hexahedra (GLL nodes, GLL points on
every quadrilateral face) and the ratio of its hex kernel time per step to the GL one.

Beside them ("batch"): 256 seeded meshes of n^3 cells (n log-uniform in [6, 40], N uniform in
2..6, c uniform in [1, 3] per layer, layers H*a | W | H*b | T | K*k) advanced by LSRK(5,4), once
mesh after mesh through dg_step and once through one dg_batch (a captured CUDA graph with one
branch per mesh); also the subset of the meshes with n <= 12.  And ("differentiation"): 400 LSRK
steps on a 32x32x40-cell mesh at N = 4 with a Ricker point source and 64 receivers, the receiver
misfit's gradient w.r.t. c^2 and the source amplitude through the checkpointed adjoint, and
central differences along 20 random c^2 directions.  And ("high_order"): the throughput mesh at
N = 5 and N = 7, single-rate LSRK, with the tet and pyramid volume products in FP32 and on the
tensor cores in split BF16 / FP16, and the modes' errors against the oracle and the exact mode.

Under torchrun (N > 1) every rank advances its own replica of the mesh (no
exchange): value = sum over ranks, time = max over ranks ("replicas only").
``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (2x2 columns of cells, all 80 layers, N = 4).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GDOF-stage/s"
ORDER = 4


def workload_config(nx, N, extra=None):
    cfg = {"workload": f"layered hybrid mesh {nx}x{nx}x80 cells, N={N}, c=1.0/1.5 by layer, upwind, "
                       "two-level multi-rate",
           "cells": [nx, nx, 80], "order": N, "l2_flush": "state 710 MB > 126 MB L2 (no flush needed)"}
    if extra:
        cfg.update(extra)
    return cfg


def sample_mesh(n):
    from paper_1507_02557_b300.inputs import layered_mesh, scale_layers
    L = scale_layers()
    return layered_mesh(n, n, len(L), L, seed=0, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)


def oracle_rate(n, steps, warmup=0, t_go=None):
    """GDOF-stage/s of the FP64 oracle on an n x n x 80 sample (this process's threads).  With
    t_go (a time.time() value) the timed steps start no earlier than t_go, so that concurrent
    processes time the same interval.  Returns (rate, ndof, seconds, start, end)."""
    from oracle.dg import DGOracle
    from paper_1507_02557_b300.inputs import random_state
    o = DGOracle(sample_mesh(n), ORDER)
    q = 1e-3 * random_state(o.ndof, 0)
    for _ in range(warmup):
        q = o.lsrk_step(q, 1e-4)
    if t_go is not None and time.time() < t_go:
        time.sleep(t_go - time.time())
    start = time.time()
    t0 = time.perf_counter()
    for _ in range(steps):
        q = o.lsrk_step(q, 1e-4)
    dt = time.perf_counter() - t0
    return o.ndof * 5 * steps / dt / 1e9, o.ndof, dt, start, time.time()


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def _oracle_children(count, n, steps, t_go, warmup=0):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_rate(%d, %d, %d, %r)))" % (ROOT, n, steps, warmup, t_go))
    procs = [subprocess.Popen([sys.executable, "-c", code], env=env, stdout=subprocess.PIPE,
                              stderr=subprocess.DEVNULL, text=True) for _ in range(count)]
    out = []
    for p in procs:
        o, _ = p.communicate(timeout=900)
        out.append(json.loads(o.strip().splitlines()[-1]))
    return out


def _oracle_children_warm(count, n, steps, warmup):
    """As _oracle_children, with warmup untimed LSRK steps in each child before the common start
    (set far enough ahead for the children's set-up and warm-up)."""
    return _oracle_children(count, n, steps, time.time() + 20.0 + 2.0 * warmup, warmup)


def cpu_baseline(n1=4, steps1=3, n_all=2, steps_all=3):
    """The oracle as it stands (FP64 numpy, one thread per process; each child is a fresh
    interpreter started as a subprocess, not a fork of this CUDA process).

    one core:  one child on an n1 x n1 x 80 sample, steps1 LSRK steps;
    all cores: nproc concurrent children, each stepping its own n_all x n_all x 80 sample (the
               oracle has no threading of its own, so the host's cores are used as independent
               processes, the way a partitioned run would use them); their timed steps start at a
               common time, and the rate is all their element-stages over the span from the first
               start to the last end."""
    one = _oracle_children(1, n1, steps1, None)[0]
    cores = os.cpu_count() or 1
    res = _oracle_children(cores, n_all, steps_all, time.time() + 20.0)
    span = max(r[4] for r in res) - min(r[3] for r in res)
    units = sum(r[1] * 5 * steps_all for r in res)
    ndof_all = res[0][1]
    return {"value": units / span / 1e9, "unit": METRIC, "cores": cores, "kind": "oracle",
            "cpu": cpu_model(), "nproc": cores,
            "sample": f"{cores} concurrent single-thread oracle processes, each {steps_all} LSRK steps on its own "
                      f"{n_all}x{n_all}x80-cell sample of the workload ({ndof_all} DOFs, N={ORDER}); "
                      f"span {span:.1f} s; FP64 numpy",
            "one_core": {"value": one[0], "unit": METRIC, "cores": 1,
                         "sample": f"{n1}x{n1}x80-cell sample ({one[1]} DOFs, N={ORDER}), {steps1} LSRK steps "
                                   f"in {one[2]:.1f} s, 1 thread"}}


class _CNvml:
    """The few read-only NVML queries the clock sampler needs, from the driver's libnvidia-ml
    through ctypes (for hosts without the Python bindings).  Constants from the public NVML API."""

    NVML_CLOCK_SM = 1
    nvmlClocksEventReasonSwPowerCap = 0x4
    nvmlClocksEventReasonHwSlowdown = 0x8
    nvmlClocksEventReasonSwThermalSlowdown = 0x20
    nvmlClocksEventReasonHwThermalSlowdown = 0x40

    def __init__(self):
        import ctypes
        self.ct = ctypes
        self.lib = ctypes.CDLL("libnvidia-ml.so.1")

    def _ok(self, rc, what):
        if rc != 0:
            raise RuntimeError(f"{what}: NVML error {rc}")

    def nvmlInit(self):
        self._ok(self.lib.nvmlInit_v2(), "nvmlInit_v2")

    def nvmlDeviceGetHandleByPciBusId(self, bus):
        h = self.ct.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByPciBusId_v2(bus.encode(), self.ct.byref(h)), "handle by bus id")
        return h

    def nvmlDeviceGetHandleByIndex(self, i):
        h = self.ct.c_void_p()
        self._ok(self.lib.nvmlDeviceGetHandleByIndex_v2(self.ct.c_uint(i), self.ct.byref(h)), "handle by index")
        return h

    def nvmlDeviceGetClockInfo(self, h, kind):
        v = self.ct.c_uint()
        self._ok(self.lib.nvmlDeviceGetClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)), "clock")
        return v.value

    def nvmlDeviceGetMaxClockInfo(self, h, kind):
        v = self.ct.c_uint()
        self._ok(self.lib.nvmlDeviceGetMaxClockInfo(h, self.ct.c_int(kind), self.ct.byref(v)), "max clock")
        return v.value

    def nvmlDeviceGetCurrentClocksEventReasons(self, h):
        v = self.ct.c_ulonglong()
        fn = getattr(self.lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            self.lib.nvmlDeviceGetCurrentClocksThrottleReasons
        self._ok(fn(h, self.ct.byref(v)), "clock event reasons")
        return v.value


class Clocks:
    """SM clock and throttle-reason sampling during the timed region: NVML queries (read-only) from
    a thread every 5 ms, so that even a region of a few tens of milliseconds gets many samples;
    nvidia-smi every 20 ms if NVML is unavailable."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, dev):
        self.dev = dev
        self.p = None
        self.thread = None
        self.samples = []          # (sm_mhz, max_mhz, set of reasons)

    def _nvml_handle(self):
        import torch
        try:
            import pynvml
        except ImportError:   # the driver's NVML library through ctypes, same read-only queries
            pynvml = _CNvml()
        pynvml.nvmlInit()
        try:
            bus = torch.cuda.get_device_properties(self.dev).pci_bus_id
            return pynvml, pynvml.nvmlDeviceGetHandleByPciBusId(bus)
        except Exception:
            return pynvml, pynvml.nvmlDeviceGetHandleByIndex(self.dev)

    def _poll(self, nv, h):
        bits = [nv.nvmlClocksEventReasonHwSlowdown, nv.nvmlClocksEventReasonHwThermalSlowdown,
                nv.nvmlClocksEventReasonSwThermalSlowdown, nv.nvmlClocksEventReasonSwPowerCap]
        mx = nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM)
        while not self.stop.is_set():
            try:
                sm = nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM)
                r = nv.nvmlDeviceGetCurrentClocksEventReasons(h)
                self.samples.append((float(sm), float(mx), {n for n, b in zip(self.NAMES, bits) if r & b}))
            except Exception:
                break
            self.stop.wait(0.005)

    def __enter__(self):
        import threading
        try:
            nv, h = self._nvml_handle()
            self.stop = threading.Event()
            self.thread = threading.Thread(target=self._poll, args=(nv, h), daemon=True)
            self.thread.start()
            return self
        except Exception as e:   # fall back to nvidia-smi, and say why
            self.thread = None
            self.nvml_error = repr(e)[:200]
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "20"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        if self.thread:
            self.stop.set()
            self.thread.join(timeout=5)
            return
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            for l in out.splitlines():
                f = [x.strip() for x in l.split(",")]
                try:
                    sm, mx = float(f[1]), float(f[2])
                except (ValueError, IndexError):
                    continue
                self.samples.append((sm, mx, {n for n, v in zip(self.NAMES, f[5:9])
                                              if v.lower().startswith("active")}))

    def summary(self):
        sm = [x[0] for x in self.samples]
        mx = [x[1] for x in self.samples]
        reasons = set().union(*[x[2] for x in self.samples]) if self.samples else set()
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(sm),
                "source": "nvml" if self.thread else "nvidia-smi",
                **({"nvml_error": self.nvml_error} if getattr(self, "nvml_error", None) else {})}


def max_over_ranks(value, dist=None, device="cpu"):
    """The largest value over all ranks (the job's time is its slowest replica's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args, rank, world):
    """The oracle on all host cores: nproc concurrent single-thread processes, each running the
    warm-up and then args.steps LSRK steps on its own 2x2x80-cell sample of the workload (timed
    steps starting at a common time); value = all their element-stages / span."""
    if rank != 0:
        return
    n = 2
    cores = os.cpu_count() or 1
    res = _oracle_children_warm(cores, n, args.steps, args.warmup)
    span = max(r[4] for r in res) - min(r[3] for r in res)
    ndof = res[0][1]
    rate = sum(r[1] * 5 * args.steps for r in res) / span / 1e9
    sample = (f"{cores} concurrent single-thread oracle processes, each {args.steps} LSRK steps (after "
              f"{args.warmup} warm-up steps) on its own {n}x{n}x80-cell sample ({ndof} DOFs, N={ORDER}); FP64 numpy")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * span / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(64, ORDER, {"sample": f"{cores} x {n}x{n}x80 cells ({ndof} DOFs each)"}),
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
                             "nproc": cores, "sample": sample},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


HEX_MRC_DRAM_BYTES_PER_ELEMENT = 879598336 / 73728   # 545,932,032 read + 333,666,304 written


def alg_bytes(t, N):
    """Algorithmic bytes of one element of type t (0 hex, 1 wedge, 2 pyramid, 3 tet) per launch
    of each kernel mode, for the data layout the kernels use: 16 B per node for each state-sized
    array moved (4 FP32 fields), 8 B per face-flux point for each trace set moved (p and u.n),
    plus the element's geometry, face data and side data (neighbour, frame code, tau: 12 B per
    face) and c^2.

    stage: fused LSRK stage (q, res read and written; traces read and written)
    trace: trace-only launch (q read, traces written)
    mrc:   fused multi-rate coarse step (q, two history slots read; rhs, q written; traces read,
           half-step and full-step traces written; the half-step set only by the coarse elements
           with a fine face neighbour, the others' total is less by one trace set, `trace_set`)
    mrf:   fused multi-rate fine substep (as mrc with one trace set written)

    Geometry: hex 21 trilinear coefficients (96 B with padding; metric terms and normals are
    recomputed); wedge 15 map coefficients (64 B with padding; the metric terms at the cubature
    points are recomputed), (n, w J^s / sqrt J) and 1 / sqrt J at its 5 (N+1)^2 face points; pyramid G, J at its semi-nodal points, (n, J^s) once
    per triangle face and (n, w J^s) at the base's points; tet G, J (12 floats) and (n, J^s) once
    per face.  Face-flux points: quad faces (N+1)^2 GL points, tet and pyramid triangle faces their
    (N+1)(N+2)/2 lattice nodes, wedge triangle faces (N+1)^2 quadrature points."""
    n1 = N + 1
    NQ, NFN = n1 * n1, n1 * (N + 2) // 2
    NP = [n1 ** 3, n1 * n1 * (N + 2) // 2, n1 * (N + 2) * (2 * N + 3) // 6, n1 * (N + 2) * (N + 3) // 6][t]
    nf = [6, 5, 5, 4][t]
    nfx = [6 * NQ, 5 * NQ, 4 * NFN + NQ, 4 * NFN][t]
    geo = [96, 64 + 5 * NQ * 16 + 5 * NQ * 4, NP * 40 + 4 * 16 + NQ * 16, 48 + 4 * 16][t]
    side = nf * 12
    st = 16 * NP
    tr = 8 * nfx
    trace_geo = [96, 5 * NQ * 4, 0, 0][t]
    return {"stage": 4 * st + 2 * tr + geo + side + 4, "trace": st + tr + trace_geo + side,
            "mrc": 5 * st + 3 * tr + geo + side + 4, "mrf": 5 * st + 2 * tr + geo + side + 4,
            "trace_set": tr}


def timed_run(g, torch, stream, steps, dt, barrier):
    """K steps inside CUDA events on the library's stream (per-type kernel timing off, so the
    element types of a stage run side by side on their own streams), then K more steps with
    per-type timing (dg_profile: one stream, CUDA events around each type's launch) for the
    per-type kernel ms, launch counts and the hex kernel's roofline."""
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    local = torch.cuda.current_device()
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        g.step(steps, dt)
        ev1.record(stream)
        barrier()
    g.profile(1)
    g.step(steps, dt)
    kms, launches = g.profile(0)
    return ev0.elapsed_time(ev1), kms, launches, clk.summary()


def batch_run(dg, torch, stream, barrier, world, steps=100, eager_steps=6, cmp_steps=30):
    """The many-mesh workload (256 meshes, 100 steps): GDOF-stage/s of per-mesh dg_step calls
    (eager, eager_steps) and of one dg_batch graph: packed (same-order meshes merged into one
    combined mesh per order: one launch per type and stage for the group; 100 steps, the workload's
    count) and unpacked (a graph branch per mesh, cmp_steps), then after the per-mesh autotuner
    (packed, cmp_steps) and the batch autotuner's pick.  Wall clock between device
    synchronisations, all meshes' states resident."""
    from paper_1507_02557_b300.inputs import batch_mesh, batch_specs, random_state
    specs = batch_specs()
    t0 = time.perf_counter()
    meshes = [dg.Mesh(batch_mesh(sp), sp[1], stream=stream.cuda_stream) for sp in specs]
    barrier()
    setup_s = time.perf_counter() - t0
    for i, g in enumerate(meshes):
        g.set_state((1e-3 * random_state(g.ndof, 100 + i)).astype(np.float32), on_device=False)
    out = {"workload": "256 meshes of n^3 cells, n log-uniform in [6,40], N uniform in 2..6, "
                       "c uniform in [1,3] per layer; LSRK(5,4)",
           "steps": steps, "setup_s": setup_s, "unit": METRIC}
    for name, sel in (("all", [True] * len(specs)), ("n_le_12", [sp[0] <= 12 for sp in specs])):
        ms = [g for g, k in zip(meshes, sel) if k]
        dof = sum(g.ndof for g in ms)
        rate = lambda n, s: dof * 5 * n * world / s / 1e9
        t1 = time.perf_counter()
        b = dg.Batch(ms, stream=stream.cuda_stream)
        barrier()
        res = {"meshes": len(ms), "dof": dof, "batch_create_s": time.perf_counter() - t1}

        def timed(f, n):
            f(3 if n >= 3 else n)       # warm-up (graph capture)
            barrier()
            t = time.perf_counter()
            f(n)
            barrier()
            return rate(n, time.perf_counter() - t)

        def eager(n):
            for g in ms:
                g.step(n)

        res["eager"] = timed(eager, eager_steps)
        res["graph"] = timed(b.step, steps)
        b.set_packing(0)
        res["graph_unpacked"] = timed(b.step, cmp_steps)
        b.set_packing(1)
        res["graph_over_eager"] = res["graph"] / res["eager"]
        res["packed_over_unpacked"] = res["graph"] / res["graph_unpacked"]
        res["graph_replays_captures"] = list(b.stats())
        t1 = time.perf_counter()
        res["batch_autotune_packed"] = b.autotune(3)
        res["batch_autotune_s"] = time.perf_counter() - t1
        b.close()
        # the same after dg_autotune picked each mesh's kernel choices (meshes whose choices now
        # differ land in different groups)
        t1 = time.perf_counter()
        picks = [g.autotune(2) for g in ms]
        res["autotune_s"] = time.perf_counter() - t1
        res["autotune_picks"] = {k: sum(p[k] for p in picks) for k in ms[0].CHOICES}
        b = dg.Batch(ms, stream=stream.cuda_stream)
        res["graph_tuned"] = timed(b.step, cmp_steps)
        b.close()
        for g in ms:
            g.set_choices()
        out[name] = res
    del meshes
    torch.cuda.synchronize()
    return out


PREC_NAMES = {0: "fp32", 1: "bf16x3", 2: "fp16x3"}


def high_order_run(dg, torch, stream, barrier, world, mesh, max_ms, steps=5):
    """The throughput mesh at N = 5 and N = 7 (75.9M / 177.8M DOFs), single-rate LSRK(5,4), with
    the tet and pyramid volume products (and at N = 7 the wedges' first contraction) in FP32 on
    the CUDA cores (precision 0) and on the tensor cores in split BF16 / FP16 (precision 1, 2):
    GDOF-stage/s and the kernel time per element type."""
    from paper_1507_02557_b300.inputs import random_state
    out = {}
    for N in (5, 7):
        res = {}
        for prec in (0, 1, 2):
            g = dg.Mesh(mesh, N, stream=stream.cuda_stream, precision=prec)
            g.set_state((1e-3 * random_state(g.ndof, 11)).astype(np.float32), on_device=False)
            dt = g.timestep()
            g.step(3, dt)
            ms, kms, _, _ = timed_run(g, torch, stream, steps, dt, barrier)
            ms = max_ms(ms)
            res[PREC_NAMES[prec]] = {"value": g.ndof * 5 * steps * world / (ms / 1e3) / 1e9, "unit": METRIC,
                                     "ms_per_step": ms / steps,
                                     "kernel_ms_per_step": {k: v / steps for k, v in
                                                            zip(["hex", "wedge", "pyramid", "tet"], kms)}}
            ndof = g.ndof
            del g
            torch.cuda.synchronize()
        res["ndof"] = ndof
        for k in ("bf16x3", "fp16x3"):
            res[k]["over_fp32"] = res[k]["value"] / res["fp32"]["value"]
        out["N%d" % N] = res
    return out


def precision_accuracy(dg, torch):
    """Errors of the three precision modes on the 4x4x5-cell hybrid mesh (c = 1) at N = 5 and 7:
    LSRK(5,4) steps from the oracle's projection of the standing mode to t = 0.01; relative L2
    difference from the FP64 oracle's state after the same steps, and the L2 error against the
    exact standing mode (the oracle's and each mode's)."""
    from oracle.dg import DGOracle, standing_mode
    from paper_1507_02557_b300.inputs import small_hybrid_mesh
    m = small_hybrid_mesh()
    out = {"workload": "4x4x5 cells HWHTK (c = 1), standing mode, LSRK(5,4) to t = 0.01", "T": 0.01}
    for N in (5, 7):
        o = DGOracle(m, N)
        q0 = o.project(standing_mode, 0.0)
        g = dg.Mesh(m, N)
        n = int(np.ceil(0.01 / g.timestep()))
        dt = 0.01 / n
        q = q0.copy()
        for _ in range(n):
            q = o.lsrk_step(q, dt)
        res = {"steps": n, "exact_l2": {"oracle_fp64": o.l2_error(q, standing_mode, 0.01)}, "oracle_rel_l2": {}}
        for prec in (0, 1, 2):
            g = dg.Mesh(m, N, precision=prec)
            g.set_state(q0.astype(np.float32), on_device=False)
            g.step(n, dt)
            got = g.get_state(np.zeros(q0.shape, np.float32), on_device=False).astype(np.float64)
            res["oracle_rel_l2"][PREC_NAMES[prec]] = float(np.linalg.norm(got - q) / np.linalg.norm(q))
            res["exact_l2"][PREC_NAMES[prec]] = o.l2_error(got, standing_mode, 0.01)
        for k in ("bf16x3", "fp16x3"):
            res[k + "_error_over_fp32"] = res["exact_l2"][k] / res["exact_l2"]["fp32"]
        out["N%d" % N] = res
    return out


def differentiation_run(dg, torch, stream, barrier, world, steps=400, every=20, ndir=20):
    """Differentiation workload: 32x32x40 cells (H*17 | W | H*19 | T | K*2), N = 4, c = 1, a Ricker
    point source (f0 = 3, t0 = 1.2/f0, amp 1) at (0, 0, -0.5), 64 receivers on an 8x8 grid of
    z = 0.8, 400 LSRK(5,4) steps of dt_min from the standing mode interpolated at the hexahedra's
    nodes; observed data from c^2 perturbed by up to 5 % per element (seeded).  Gradient of
    1/2 sum (d - d_obs)^2 w.r.t. c^2 and amp through autograd.Seismogram (checkpoints every 20
    steps); dL/dc^2 checked against central differences of forward runs along ndir random
    directions (relative step 1e-3)."""
    import dataclasses

    from paper_1507_02557_b300.autograd import seismogram
    from paper_1507_02557_b300.inputs import layered_mesh
    layers = "H" * 17 + "W" + "H" * 19 + "T" + "K" * 2
    mesh = layered_mesh(32, 32, 40, layers, seed=0)
    g1 = np.linspace(-0.75, 0.75, 8)
    recs = [[x, y, 0.8] for y in g1 for x in g1]
    f0 = 3.0
    rng = np.random.default_rng(5)

    def make(c2, amp=1.0):
        g = dg.Mesh(dataclasses.replace(mesh, c2=c2), ORDER, stream=stream.cuda_stream)
        g.set_source([0.0, 0.0, -0.5], amp, f0, 1.2 / f0)
        g.set_receivers(recs)
        return g

    g = make(mesh.c2)
    dt = g.timestep()
    nel = sum(mesh.nelem)
    # initial state: the standing mode's p at the hexahedra's GL nodes (trilinear maps), 0 elsewhere
    x, _ = np.polynomial.legendre.leggauss(ORDER + 1)
    n1 = ORDER + 1
    idx = np.arange(n1 ** 3)
    rst = np.stack([x[idx % n1], x[(idx // n1) % n1], x[idx // n1 ** 2]], 1)
    corner = np.array([[(-1) ** (1 + (v & 1)), (-1) ** (1 + ((v >> 1) & 1)), (-1) ** (1 + ((v >> 2) & 1))]
                       for v in range(8)], float)
    shape = np.prod(1 + rst[:, None, :] * corner[None, :, :], axis=2) / 8
    X = torch.einsum("nv,kvd->knd", torch.from_numpy(shape).cuda(), torch.from_numpy(mesh.xyz[mesh.conn[0]]).cuda())
    q0 = torch.zeros((4, g.ndof), dtype=torch.float32, device="cuda")
    p0 = torch.cos(np.pi / 2 * X[..., 0]) * torch.cos(np.pi / 2 * X[..., 1]) * torch.cos(np.pi / 2 * X[..., 2])
    q0[0, :p0.numel()] = p0.reshape(-1).float()
    zeros = lambda n: torch.zeros(n, dtype=torch.float64, device="cuda")
    go = make([c * (1 + 0.05 * rng.uniform(-1, 1, len(c))) for c in mesh.c2])
    with torch.no_grad():
        obs = seismogram(go, q0, zeros(nel), zeros(1), steps, dt, 0.0, every).double()
    del go

    def loss(gm, grad=False):
        c2 = zeros(nel).requires_grad_(grad)
        amp = zeros(1).requires_grad_(grad)
        d = seismogram(gm, q0, c2, amp, steps, dt, 0.0, every)
        return 0.5 * ((d.double() - obs) ** 2).sum(), c2, amp

    Lw, _, _ = loss(g, True)          # warm-up (first use of the loss's torch kernels, adjoint scratch)
    Lw.backward()
    barrier()
    t0 = time.perf_counter()
    L, c2, amp = loss(g, True)
    barrier()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    L.backward()
    barrier()
    t_bwd = time.perf_counter() - t0
    gc = c2.grad.cpu().numpy()
    c2all = np.concatenate(mesh.c2)
    errs = []
    for _ in range(ndir):
        dirs = rng.standard_normal(nel)
        parts = np.split(dirs, np.cumsum(mesh.nelem)[:-1])
        lp = float(loss(make([c * (1 + 1e-3 * d_) for c, d_ in zip(mesh.c2, parts)]))[0])
        lm = float(loss(make([c * (1 - 1e-3 * d_) for c, d_ in zip(mesh.c2, parts)]))[0])
        fd = (lp - lm) / 2e-3
        ad = float(np.sum(gc * c2all * dirs))
        errs.append(abs(fd - ad) / max(abs(ad), 1e-300))
    lp = float(loss(make(mesh.c2, 1.0 + 1e-3))[0])
    lm = float(loss(make(mesh.c2, 1.0 - 1e-3))[0])
    units = g.ndof * 5 * steps * world
    out = {"workload": "32x32x40 cells (H*17|W|H*19|T|K*2), N=4, Ricker source at (0,0,-0.5), 64 receivers "
                       "at z=0.8, %d LSRK(5,4) steps of dt_min, checkpoints every %d" % (steps, every),
           "ndof": g.ndof, "dt": dt, "loss": float(L.detach()), "unit": METRIC,
           "forward": units / t_fwd / 1e9, "backward": units / t_bwd / 1e9, "backward_over_forward": t_bwd / t_fwd,
           "fd_directions": ndir, "fd_rel_err_max": max(errs), "fd_rel_err_median": float(np.median(errs)),
           "grad_amp": float(amp.grad.item()), "grad_amp_fd": (lp - lm) / 2e-3,
           "grad_amp_note": "within the window the source's signal (speed <= 1.5, 0.046 time units) "
                            "cannot reach the z=0.8 plane 1.3 away: dL/damp is 0 up to the scheme's "
                            "exponentially small leakage, and the central difference is FP32 rounding "
                            "of L divided by 2e-3"}
    del g
    torch.cuda.synchronize()
    return out


def run_case(args, dg, torch, mesh):
    """--case: warm-up steps, then the timed steps (lsrk) or one adjoint window (adjoint); one JSON
    line with the wall time (not a bench value)."""
    from paper_1507_02557_b300.inputs import random_state
    g = dg.Mesh(mesh, args.order, precision=args.precision, nlevels=args.nlevels)
    g.set_state((1e-3 * random_state(g.ndof, 1)).astype(np.float32), on_device=False)
    dt = g.timestep()
    g.step(args.warmup, dt)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.case == "lsrk":
        g.step(args.steps, dt)
    else:
        lam = torch.from_numpy(random_state(g.ndof, 2).astype(np.float32)).cuda()
        grad = torch.zeros(sum(mesh.nelem), dtype=torch.float64, device="cuda")
        g.adjoint_step(args.steps, lam, grad, dt)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "order": args.order, "cells": args.cells, "ndof": g.ndof,
                      "precision": args.precision, "nlevels": args.nlevels,
                      "steps": args.steps, "wall_s": time.perf_counter() - t0}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cells", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the differentiation and high-order lines")
    ap.add_argument("--case", choices=["lsrk", "adjoint"], default=None,
                    help="run one small case only (for profiling): LSRK steps at --order, or one adjoint "
                         "window of --steps steps with the c^2 gradient, on the --cells x --cells x 80 mesh")
    ap.add_argument("--order", type=int, default=ORDER)
    ap.add_argument("--precision", type=int, default=0, help="--case: 0 FP32, 1 BF16 x 3, 2 FP16 x 3 products")
    ap.add_argument("--nlevels", type=int, default=1, help="--case lsrk: 1 single rate, 2 multi-rate AB3")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_1507_02557_b300 import dg
    from paper_1507_02557_b300.inputs import random_state, scale_mesh
    import json

    mesh = scale_mesh(args.cells, args.cells)
    if args.case:
        return run_case(args, dg, torch, mesh)
    stream = torch.cuda.current_stream()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    K_hex = mesh.nelem[0]
    ab = [alg_bytes(t, ORDER) for t in range(4)]
    hb = ab[0]
    TYPES = ["hex", "wedge", "pyramid", "tet"]

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    def max_ms(ms):
        return max_over_ranks(ms, dist, "cuda")

    # ---- single-rate LSRK(5,4): fused stage kernels
    g1 = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream, nlevels=1)
    ndof = g1.ndof
    q0 = (1e-3 * random_state(ndof, 1 + rank)).astype(np.float32)
    g1.set_state(q0, on_device=False)
    dt = g1.timestep()
    g1.step(args.warmup, dt)
    ms1, kms1, l1, clk1 = timed_run(g1, torch, stream, args.steps, dt, barrier)
    ms1 = max_ms(ms1)
    n_stage = 5 * args.steps
    # per type: n_stage fused stage launches and the trace launch of the dg_step call
    tb1 = [mesh.nelem[t] * (ab[t]["stage"] * n_stage + ab[t]["trace"] * (l1[t] - n_stage)) if l1[t] else 0
           for t in range(4)]
    hex_bytes1 = tb1[0]
    ach1 = hex_bytes1 / (kms1[0] / 1e3) / 1e9
    step1 = sum(tb1) / (ms1 / 1e3) / 1e9
    single = {"value": ndof * 5 * args.steps * world / (ms1 / 1e3) / 1e9, "unit": METRIC,
              "ms_per_step": ms1 / args.steps, "integrator": "LSRK(5,4), 5 stages per step",
              "kernel_ms": dict(zip(TYPES, kms1)),
              "kernel_gbs": {n: (b / (k / 1e3) / 1e9 if k > 0 else None) for n, b, k in zip(TYPES, tb1, kms1)},
              "hex_stage_kernel": {"achieved": ach1, "peak": hbm, "unit": "GB/s", "frac": ach1 / hbm},
              "step_roofline": {"bytes_per_step": sum(tb1) / args.steps, "achieved": step1, "peak": hbm,
                                "unit": "GB/s", "frac": step1 / hbm},
              "gpu_launches": int(sum(l1))}
    # the same steps with the warp-per-element SIMT tet kernel instead of the tensor-core one
    g1.set_choices(tet_tensor_cores=False)
    g1.profile(1)
    g1.step(args.steps, dt)
    kms_simt, _ = g1.profile(0)
    g1.set_choices()
    single["tet_tensor_cores_vs_simt"] = {"tensor_core_ms": kms1[3], "simt_ms": kms_simt[3],
                                          "time_ratio": kms1[3] / kms_simt[3] if kms_simt[3] > 0 else None,
                                          "note": "tet kernel time over the same LSRK steps (per-type timing)"}
    del g1
    torch.cuda.synchronize()

    # ---- two-level multi-rate AB3 (the workload as specified): headline
    g = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream, nlevels=2)
    g.set_state(q0, on_device=False)
    h = g.timestep()
    fine = g.level_type_counts(2)
    npe = [(ORDER + 1) ** 3, (ORDER + 1) ** 2 * (ORDER + 2) // 2,
           (ORDER + 1) * (ORDER + 2) * (2 * ORDER + 3) // 6, (ORDER + 1) * (ORDER + 2) * (ORDER + 3) // 6]
    ndof_fine = sum(c * n for c, n in zip(fine, npe))
    g.step(args.warmup, h)                                   # includes the LSRK start-up
    E_before = g.energy()                                    # synchronises; outside the timed region
    ms, kms, launches, clk = timed_run(g, torch, stream, args.steps, h, barrier)
    E_after = g.energy()                                     # after the timed and the profiled steps
    ms = max_ms(ms)
    stage_units = (ndof + ndof_fine) * args.steps * world    # rhs evaluations actually performed
    value = stage_units / (ms / 1e3) / 1e9
    # hex kernels: one trace launch per dg_step call, then per coarse step the fused coarse
    # step of the coarse hexes and two fused substeps of the fine hexes
    iface = g.level_type_counts(-1)   # coarse elements with a fine neighbour: they alone write half-step traces
    tb = [mesh.nelem[t] * ab[t]["trace"] + args.steps * ((mesh.nelem[t] - fine[t]) * ab[t]["mrc"]
                                                         - (mesh.nelem[t] - fine[t] - iface[t]) * ab[t]["trace_set"]
                                                         + 2 * fine[t] * ab[t]["mrf"]) for t in range(4)]
    hex_bytes = tb[0]
    achieved = hex_bytes / (kms[0] / 1e3) / 1e9
    # whole step: the algorithmic bytes of every kernel of the timed steps over the timed region
    step_gbs = sum(tb) / (ms / 1e3) / 1e9
    # DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one launch of the TMA-staged
    # hexw_kernel<4,MRC>, measured with ncu on the 32x32x80-cell mesh (73,728 hexahedra) and
    # scaled by the elements of one full-size launch
    traffic = HEX_MRC_DRAM_BYTES_PER_ELEMENT * (K_hex - fine[0])
    # end to end through the public API with host buffers: one simulation call = H2D of the
    # state from pinned host memory, K coarse steps (the first call after dg_set_state also runs
    # the LSRK start-up of the history: 4 LSRK steps + 3 rhs, counted as performed stages),
    # D2H of the final state into pinned host memory
    pinned = torch.from_numpy(q0).pin_memory()
    out_h = torch.empty_like(pinned).pin_memory()
    barrier()
    t0 = time.perf_counter()
    g.set_state(pinned, on_device=False)
    g.step(args.steps, h)
    g.get_state(out_h, on_device=False)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_units = ((ndof + ndof_fine) * args.steps + 23 * ndof) * world
    e2e = {"value": e2e_units / e2e_s / 1e9, "unit": METRIC,
           "h2d_bytes_per_step": 4 * ndof * 4 / args.steps, "d2h_bytes_per_step": 4 * ndof * 4 / args.steps,
           "steps": args.steps,
           "note": "one public-API call sequence: dg_set_state(host) + dg_step(K) + dg_get_state(host), "
                   "including the history start-up; copies amortised over the K steps"}
    # per step re-upload (single-rate path has no history): H2D state + 1 LSRK step + energy to host
    g1 = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream, nlevels=1)
    barrier()
    t0 = time.perf_counter()
    e_steps = max(3, min(args.steps, 20))
    for _ in range(e_steps):
        g1.set_state(pinned, on_device=False)
        g1.step(1, dt)
        g1.energy()
    barrier()
    e2 = time.perf_counter() - t0
    single["e2e_per_step_upload"] = {"value": ndof * 5 * e_steps * world / e2 / 1e9, "unit": METRIC,
                                     "h2d_bytes_per_step": 4 * ndof * 4, "d2h_bytes_per_step": 8}
    del g1

    # ---- multi-rate LSRK(5,4) (integrator 1) on the same workload, beside MRAB3: per coarse step
    # five full rhs evaluations (z_j = B^j y), five on S (u_j) and ten on S (the fine correction's
    # stages), S = fine elements and the coarse elements next to them
    mr_lsrk = None
    if not args.no_extras:
        gl = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream, nlevels=2, integrator=1)
        gl.set_state(q0, on_device=False)
        s_count = gl.mr_s_counts()
        ndof_s = sum(c * n for c, n in zip(s_count, npe))
        l_steps = max(3, min(args.steps, 10))
        gl.step(args.warmup, h)
        ms_l, kms_l, _, _ = timed_run(gl, torch, stream, l_steps, h, barrier)
        ms_l = max_ms(ms_l)
        mr_lsrk = {"value": (5 * ndof + 15 * ndof_s) * l_steps * world / (ms_l / 1e3) / 1e9, "unit": METRIC,
                   "steps": l_steps, "ms_per_coarse_step": ms_l / l_steps, "ndof_S": ndof_s,
                   "kernel_ms": dict(zip(TYPES, kms_l)),
                   "time_per_simulated_time_over_mrab3": (ms_l / l_steps) / (ms / args.steps),
                   "note": "value counts the rhs element evaluations performed (5 full + 15 on S per coarse step); "
                           "the ratio compares wall time per coarse step 2h with the MRAB3 headline"}
        del gl
        torch.cuda.synchronize()

    # ---- SEM hexahedra (GLL nodes, GLL points on quad faces): the same multi-rate workload, for
    # the cost comparison of the two hex bases (per-DOF time of the hex kernels)
    del g
    torch.cuda.synchronize()
    gs = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream, nlevels=2, hex_basis=1)
    gs.set_state(q0, on_device=False)
    hs = gs.timestep()
    fs = gs.level_type_counts(2)
    ndof_fine_s = sum(c * n for c, n in zip(fs, npe))
    s_steps = max(3, min(args.steps, 20))
    gs.step(args.warmup, hs)
    ms_s, kms_s, _, _ = timed_run(gs, torch, stream, s_steps, hs, barrier)
    ms_s = max_ms(ms_s)
    sem = {"value": (ndof + ndof_fine_s) * s_steps * world / (ms_s / 1e3) / 1e9, "unit": METRIC,
           "steps": s_steps, "ms_per_step": ms_s / s_steps, "h_fine": hs, "fine_elements": fs,
           "kernel_ms": dict(zip(["hex", "wedge", "pyramid", "tet"], kms_s)),
           "hex_time_sem_over_gl": (kms_s[0] / s_steps) / (kms[0] / args.steps)}
    del gs
    torch.cuda.synchronize()
    batch = None if args.no_batch else batch_run(dg, torch, stream, barrier, world)
    diff = None if args.no_extras else differentiation_run(dg, torch, stream, barrier, world)
    high = None if args.no_extras else high_order_run(dg, torch, stream, barrier, world, mesh, max_ms)
    if high and rank == 0:
        high["accuracy"] = precision_accuracy(dg, torch)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.cells, ORDER, {
                    "integrator": "two-level multi-rate AB3 (step = one coarse step of 2h)",
                    "ndof": ndof, "ndof_fine": ndof_fine, "elements": mesh.nelem, "fine_elements": fine, "coarse_elements_with_fine_neighbour": iface,
                    "h_fine": h, "parallelism": "replicas" if world > 1 else "single GPU"}),
                "roofline": {"bound": "hbm", "kernel": "hexw_kernel<4,MRC> (fused multi-rate coarse step)",
                             "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                             "traffic": traffic, "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)",
                             "step": {"bytes_per_step": sum(tb) / args.steps, "achieved": step_gbs, "peak": hbm,
                                      "unit": "GB/s", "frac": step_gbs / hbm,
                                      "note": "algorithmic bytes of all kernels of the timed steps (every type "
                                              "and mode, alg_bytes) / ms_per_step"}},
                "kernel_ms": dict(zip(TYPES, kms)),
                "kernel_gbs": {n: (b / (k / 1e3) / 1e9 if k > 0 else None) for n, b, k in zip(TYPES, tb, kms)},
                "gpu_launches": int(sum(launches)) + 2 * 4 * args.steps,
                "single_rate": single, "sem_hex": sem, "mr_lsrk": mr_lsrk, "e2e": e2e, "clocks": clk,
                "energy": {"before": E_before, "after": E_after, "rel_change": (E_after - E_before) / E_before,
                           "note": "discrete energy before and after the timed and the profiled multi-rate steps (upwind: non-increasing)"}}
        if batch:
            line["batch"] = batch
        if diff:
            line["differentiation"] = diff
        if high:
            line["high_order"] = high
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
