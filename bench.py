"""Throughput benchmark: GDOF-stage/s of the hybrid-mesh DG right-hand side + LSRK(5,4) stage.

Workload: the 64x64x80-cell layered hybrid mesh on [-1,1]^3 (layers
H x34 | W x2 | H x36 | T | K x4 | U | H x2: 294,912 hex, 16,384 wedges, 40,960
pyramids, 114,688 tets), order N = 4 (44,359,680 DOFs x 4 fields), wave speed
1.0 / 1.5 alternating by layer, upwind flux.  One step = one LSRK(5,4) step (five
right-hand-side evaluations and stage updates) over the whole mesh, all element
types.  GDOF-stage/s = ndof * 5 * steps / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl b300|reference]

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
                       "LSRK(5,4) single-rate",
           "cells": [nx, nx, 80], "order": N, "l2_flush": "state 710 MB > 126 MB L2 (no flush needed)"}
    if extra:
        cfg.update(extra)
    return cfg


def sample_mesh(n):
    from paper_1507_02557_b300.inputs import layered_mesh, scale_layers
    L = scale_layers()
    return layered_mesh(n, n, len(L), L, seed=0, c_of_layer=lambda k: 1.0 if k % 2 == 0 else 1.5)


def oracle_rate(n, steps, warmup=0):
    """GDOF-stage/s of the FP64 oracle on an n x n x 80 sample (this process's threads)."""
    from oracle.dg import DGOracle
    from paper_1507_02557_b300.inputs import random_state
    o = DGOracle(sample_mesh(n), ORDER)
    q = 1e-3 * random_state(o.ndof, 0)
    for _ in range(warmup):
        q = o.lsrk_step(q, 1e-4)
    t0 = time.perf_counter()
    for _ in range(steps):
        q = o.lsrk_step(q, 1e-4)
    dt = time.perf_counter() - t0
    return o.ndof * 5 * steps / dt / 1e9, o.ndof, dt


def cpu_baseline(n=4, steps=3):
    """Run the oracle in a single-threaded child process on an n x n x 80 sample."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "r = bench.oracle_rate(%d, %d); print(json.dumps(r))" % (ROOT, n, steps))
    out = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True, timeout=900)
    rate, ndof, secs = json.loads(out.stdout.strip().splitlines()[-1])
    return {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"{n}x{n}x80-cell sample of the workload ({ndof} DOFs, N={ORDER}), "
                      f"{steps} LSRK steps in {secs:.1f} s, FP64 numpy, 1 thread"}


class Clocks:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev):
        self.dev = dev
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.p:
            self.p.terminate()
            try:
                out, _ = self.p.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.p.kill()
                out, _ = self.p.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons), "samples": len(sm)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    n = 2
    rate, ndof, secs = oracle_rate(n, args.steps, args.warmup)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(64, ORDER, {"sample": f"{n}x{n}x80 cells ({ndof} DOFs)"}),
            "cpu_baseline": {"value": rate, "unit": METRIC, "cores": 1, "kind": "oracle",
                             "sample": f"{n}x{n}x80-cell sample ({ndof} DOFs), {args.steps} LSRK steps"},
            "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def hex_alg_bytes(N):
    """Algorithmic bytes of one hex element in the fused stage kernel and the trace kernel."""
    NP, NQ = (N + 1) ** 3, (N + 1) ** 2
    stage = 4 * NP * 4 * 4 + 96 + 4 + 6 * 12 + 2 * 6 * NQ * 8   # q,res r/w; geometry; c2; sides; traces r+w
    trace = 4 * NP * 4 + 96 + 6 * 12 + 6 * NQ * 8
    return stage, trace


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="b300", choices=["b300", "reference"])
    ap.add_argument("--cells", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
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

    mesh = scale_mesh(args.cells, args.cells)
    stream = torch.cuda.current_stream()
    g = dg.Mesh(mesh, ORDER, stream=stream.cuda_stream)
    ndof = g.ndof
    q0 = (1e-3 * random_state(ndof, 1 + rank)).astype(np.float32)
    g.set_state(q0, on_device=False)
    dt = g.timestep()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up, then K timed steps (one dg_step call), per-type kernel events on the same stream
    g.step(args.warmup, dt)
    barrier()
    g.profile(1)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        barrier()
        ev0.record(stream)
        g.step(args.steps, dt)
        ev1.record(stream)
        barrier()
    ms = ev0.elapsed_time(ev1)
    kms, launches = g.profile(0)
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    stage_units = ndof * 5 * args.steps * world
    value = stage_units / (ms / 1e3) / 1e9

    # dominant kernel roofline: the hexahedron stage kernel
    import json as _json
    peaks = {}
    try:
        peaks = _json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    K_hex = mesh.nelem[0]
    b_stage, b_trace = hex_alg_bytes(ORDER)
    n_stage = 5 * args.steps
    n_trace = launches[0] - n_stage
    hex_bytes = K_hex * (b_stage * n_stage + b_trace * n_trace)
    achieved = hex_bytes / (kms[0] / 1e3) / 1e9
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "hex_stage_traffic.json")
    if os.path.exists(tfile):
        try:
            traffic = _json.load(open(tfile)).get("bytes_per_launch")
        except (OSError, ValueError):
            traffic = None

    # end to end through the public API: per step, H2D of the state from pinned host memory,
    # one LSRK step, and the step's energy read back to the host
    pinned = torch.from_numpy(q0).pin_memory()
    barrier()
    t0 = time.perf_counter()
    e_steps = max(3, min(args.steps, 20))
    for _ in range(e_steps):
        g.set_state(pinned, on_device=False)
        g.step(1, dt)
        g.energy()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": ndof * 5 * e_steps * world / e2e_s / 1e9, "unit": METRIC,
           "h2d_bytes_per_step": 4 * ndof * 4, "d2h_bytes_per_step": 8, "steps": e_steps}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": workload_config(args.cells, ORDER, {
                    "ndof": ndof, "elements": mesh.nelem, "dt": dt,
                    "parallelism": "replicas" if world > 1 else "single GPU"}),
                "roofline": {"bound": "hbm", "kernel": "hex_kernel<4,STAGE>", "achieved": achieved,
                             "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": traffic,
                             "alg_bytes_per_launch": K_hex * b_stage,
                             "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)"},
                "kernel_ms": dict(zip(["hex", "wedge", "pyramid", "tet"], kms)),
                "gpu_launches": int(sum(launches)),
                "e2e": e2e, "clocks": clk.summary()}
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
