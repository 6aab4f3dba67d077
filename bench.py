#!/usr/bin/env python
"""Benchmark of the depth march: phase-space cell-updates per second.

One bench step is one depth step h of the whole hot path (E(h/2) T(h/2) A(h)
T(h/2) E(h/2) on every component) over the 150 MeV pencil beam in water on a
128x128 lateral grid (1 mm), 256 energy groups over 0-160 MeV and 16x16 angles
in +-0.15 rad, psi in FP32 (the single-GPU workload the metric is quoted on).
A cell is one (y, z, E-group, u, v) point with both DG coefficients; a
cell-update is one cell advanced by one depth step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank marches its own beam (independent pencil
beams: weak scaling, no data-path collective); the time is the maximum over
ranks and the value counts the cell-updates of all ranks.  Rank 0 prints one
JSON line.  --impl reference times the FP64 CPU oracle on the host cores on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "phase-space cell-updates/s (mixed vs FP64, same GB300, dose err\u22641e-3); % HBM peak"
UNIT = "cell-updates/s"


def _args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=60)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-fp64", action="store_true", help="skip the FP64-GPU comparison run")
    p.add_argument("--no-cpu-baseline", action="store_true", help="skip the CPU-oracle baseline")
    return p.parse_args()


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    Q = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = bus_id
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        if self.bus_id:
            mine = [r for r in rows if len(r) >= 10 and self.bus_id.lower() in r[1].lower()]
            rows = mine or rows
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            if len(r) < 10:
                continue
            try:
                sm.append(float(r[2]))
                mx.append(float(r[3]))
            except ValueError:
                continue
            for n, v in zip(names, r[6:10]):
                if v.strip().lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- roofline helpers

def _kernel_hash(names) -> str:
    h = hashlib.sha256()
    for name in names:
        with open(os.path.join(ROOT, "paper_2504_00340_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


# the source files of each kernel (its .cu and the device code it includes)
KERNEL_FILES = {"energy": ("k_energy_f2.cu", "energy_f2.cuh"),
                "transport": ("k_transport_rows.cu", "transport_rows.cuh"),
                "angular": ("k_angular.cu", "angular_f2.cuh"), "source": ("k_source_tc.cu",)}


def _traffic_from_profiles(kind: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary of this kernel and
    workload, if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", f"{kind}_{workload}.md")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        text = f.read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", text)
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", text)
    if not m or not h or h.group(1) != _kernel_hash(KERNEL_FILES[kind]):
        return None
    return float(m.group(1))


# ---------------------------------------------------------------- our arm

def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist
    from paper_2504_00340_gb300 import binding
    from paper_2504_00340_gb300.workloads import WATER150

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    def barrier():
        if world > 1:
            dist.barrier()

    # CPU baseline first, before this process starts its GPU work (rank 0, N = 1)
    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        cpu = cpu_baseline_sample(budget_s=15.0)

    w = WATER150
    grid = w.grid()
    W, K = a.warmup, a.steps
    nx = W + K
    rho = np.ones((nx, w.ny, w.nz))
    cells = w.cells_per_step * (w.n_scatter + 1)
    stream = torch.cuda.current_stream()
    s = binding.Solver(grid, nx=nx, dx=w.dx, n_scatter=w.n_scatter, precision="fp32", stream=stream)
    s.set_material(rho)
    s.launch_beam(**w.beam)
    # launch shapes and kernel forms from the library's autotuner (restarts the beam)
    s.autotune(4)
    tuning = s.tuning
    s.step(W)
    s.flush()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    bus = None
    for attr in ("pci_bus_id",):
        v = getattr(props, attr, None)
        if isinstance(v, int):
            bus = f"{v:02x}:"
    sampler = ClockSampler(bus)
    time.sleep(0.5)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    l0 = s.kernel_launches
    s.set_profiling(True)
    ev0.record(stream)
    s.step(K)
    s.flush()  # the deferred closing half step of the last timed step
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = s.kernel_launches - l0
    prof = s.profile()
    s.set_profiling(False)
    if world > 1:
        t = torch.tensor([ms], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    total_cells = cells * K * world
    value = total_cells / (ms / 1e3)

    # roofline of the dominant kernel: algorithmic bytes = one read + one write
    # of both FP32 DG coefficients of every cell of every component it updates
    bytes_per_launch = {"energy": cells * 2 * 4 * 2, "transport": cells * 2 * 4 * 2,
                        "angular": cells * 2 * 4 * 2, "source": None}
    dom = max((k for k in prof if prof[k][0] > 0), key=lambda k: prof[k][1])
    n_l, t_ms = prof[dom]
    avg_s = t_ms / n_l / 1e3
    peak, peak_kind = _peaks()
    achieved = bytes_per_launch[dom] / avg_s / 1e9
    roofline = {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "peak_source": peak_kind,
                "bytes_per_launch": bytes_per_launch[dom], "avg_launch_ms": round(avg_s * 1e3, 4),
                "traffic": _traffic_from_profiles(dom, "water150")}
    kernels = {k: {"launches": v[0], "total_ms": round(v[1], 3),
                   "avg_ms": round(v[1] / v[0], 4) if v[0] else None,
                   "hbm_frac": (round(bytes_per_launch[k] / (v[1] / v[0] / 1e3) / 1e9 / peak, 4)
                                if v[0] and bytes_per_launch[k] else None)}
               for k, v in prof.items() if v[0]}
    s.close()
    del s
    torch.cuda.empty_cache()

    # end to end through the public API with host buffers: material in,
    # beam projection, K steps, dose out (the copies are inside the region)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = binding.Solver(grid, nx=K, dx=w.dx, n_scatter=w.n_scatter, precision="fp32", stream=stream)
    s.set_tuning(**tuning)
    s.set_material(rho[:K])
    s.launch_beam(**w.beam)
    s.step(K)
    dose = s.read_dose(K)
    t1 = time.perf_counter()
    s.close()
    del s
    torch.cuda.empty_cache()
    e2e_s = t1 - t0
    if world > 1:
        t = torch.tensor([e2e_s], device="cuda", dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    nyz = w.ny * w.nz
    h2d = K * nyz * 4 + (2 * w.ng + w.na + w.ny + w.nz) * 8
    d2h = K * nyz * 8
    e2e = {"value": cells * K * world / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d / K,
           "d2h_bytes_per_step": d2h / K,
           "includes": "context + workspace allocation, material upload, beam projection, K steps, dose readback"}

    # FP64 GPU form on the same workload (a few steps), and the FP32 dose error against it
    fp64 = None
    if rank == 0 and not a.no_fp64:
        fp64 = fp64_comparison(binding, w, stream, n=4)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
            "ms_per_step": ms / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": w.name, "beam": "150 MeV, sigma_y=sigma_z=0.4 cm, sigma_E=1 MeV, water",
                       "lateral": "128x128 @ 1 mm", "energy_groups": "256 over 0-160 MeV",
                       "angles": "16x16 in +-0.15 rad", "dx_cm": w.dx, "components": w.n_scatter + 1,
                       "precision": "fp32 psi, fp64 dose tally",
                       "cells_per_step_per_gpu": cells, "parallelism": f"replicas x{world} (independent beams)",
                       "l2": "inputs larger than L2: psi is 8.6 GB per GPU"},
            "roofline": roofline,
            "kernels": kernels,
            "tuning": tuning,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
            "fp64_gpu": fp64,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def _march_dose(binding, w, grid, nx, prec, stream, timed=False):
    """March nx depth steps of workload w on grid in one precision; returns
    (cell-updates/s or None, dose [s][y][z], fluence [s][y][z])."""
    import numpy as np
    import torch
    s = binding.Solver(grid, nx=nx, dx=w.dx, n_scatter=w.n_scatter, precision=prec, stream=stream)
    s.set_material(np.ones((nx, grid["ny"], grid["nz"])))
    s.launch_beam(**w.beam)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(nx)
    s.flush()
    e1.record(stream)
    torch.cuda.synchronize()
    cells = grid["ny"] * grid["nz"] * (len(grid["e_faces"]) - 1) * grid["nu"] * grid["nv"] * (w.n_scatter + 1)
    rate = cells * nx / (e0.elapsed_time(e1) / 1e3) if timed else None
    dose, flu = s.read_dose(nx), s.read_fluence(nx + 1)
    s.close()
    del s
    torch.cuda.empty_cache()
    return rate, dose, flu


def fp64_comparison(binding, w, stream, n=4, lateral=32):
    """The FP64 GPU form of the workload: its speed on the full grid over the
    first n steps, and the FP32 dose and fluence error against it over the
    whole depth (all of the workload's steps, through the Bragg peak) on a
    reduced lateral grid with the workload's own energy and angle grids."""
    import numpy as np
    grid = w.grid()
    rate64, d64, _ = _march_dose(binding, w, grid, n, "fp64", stream, timed=True)
    rate32, d32, _ = _march_dose(binding, w, grid, n, "fp32", stream, timed=True)
    small = dict(grid, ny=lateral, nz=lateral)
    _, fd64, ff64 = _march_dose(binding, w, small, w.n_steps, "fp64", stream)
    _, fd32, ff32 = _march_dose(binding, w, small, w.n_steps, "fp32", stream)
    idd = fd64.sum(axis=(1, 2))
    return {"value": rate64, "unit": UNIT, "steps": n,
            "fp32_speedup": rate32 / rate64,
            "dose_err_fp32_vs_fp64_entrance": float(np.abs(d32 - d64).max() / np.abs(d64).max()),
            "full_depth": {
                "lateral": f"{lateral}x{lateral} @ {w.dy * 10:g} mm", "steps": w.n_steps,
                "depth_cm": w.n_steps * w.dx,
                "bragg_peak_cm": float((np.argmax(idd) + 0.5) * w.dx),
                "dose_err_fp32_vs_fp64": float(np.abs(fd32 - fd64).max() / np.abs(fd64).max()),
                "fluence_err_fp32_vs_fp64": float(np.abs(ff32 - ff64).max() / np.abs(ff64).max())},
            "note": (f"speed: the full workload grid, first {n} steps; error: every step of the workload's depth on a "
                     f"{lateral}x{lateral} lateral grid with its 256 groups and 16x16 angles (max-normalised)")}


# ---------------------------------------------------------------- CPU oracle

def _oracle_sample(n_groups):
    """The benchmark workload restricted to its top n_groups energy groups
    (the ones holding the beam), full lateral grid and angles."""
    import numpy as np
    import oracle
    from paper_2504_00340_gb300.workloads import WATER150
    w = WATER150
    grid = dict(w.grid())
    grid["e_faces"] = w.e_faces[-(n_groups + 1):]
    o = oracle.Oracle(grid)
    psi = o.init_beam(w.beam)[None]
    return o, psi, np.ones((1, w.ny, w.nz)), w


def cpu_baseline_sample(budget_s=15.0, n_groups=16):
    """Time the oracle as it stands on a bounded sample (about budget_s of CPU work)."""
    import oracle
    o, psi, rho, w = _oracle_sample(n_groups)
    cells = w.ny * w.nz * n_groups * w.na
    steps, t = 0, 0.0
    while t < budget_s and steps < 20:
        t0 = time.perf_counter()
        psi = o.march(rho, 1, w.dx, psi=psi)["psi"]
        t += time.perf_counter() - t0
        steps += 1
    return {"value": cells * steps / t, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"{steps} depth steps of the top {n_groups} of 256 groups, full 128x128 lateral, 16x16 angles "
                      f"(FP64 C oracle, OpenMP), {t:.1f} s"}


def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return
    import oracle
    # size the per-step sample so that warmup + steps take about 150 s in all
    o, psi, rho, w = _oracle_sample(4)
    t0 = time.perf_counter()
    o.march(rho, 1, w.dx, psi=psi)
    per_group = (time.perf_counter() - t0) / 4
    budget = 150.0 / max(1, a.steps + a.warmup)
    ng = int(max(1, min(256, budget / max(per_group, 1e-6))))
    o, psi, rho, w = _oracle_sample(ng)
    cells = w.ny * w.nz * ng * w.na
    for _ in range(a.warmup):
        psi = o.march(rho, 1, w.dx, psi=psi)["psi"]
    t0 = time.perf_counter()
    for _ in range(a.steps):
        psi = o.march(rho, 1, w.dx, psi=psi)["psi"]
    t = time.perf_counter() - t0
    value = cells * a.steps / t
    sample = (f"each step: one depth step of the top {ng} of 256 groups, full 128x128 lateral, 16x16 angles "
              f"(FP64 C oracle, OpenMP)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t / a.steps * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    args = _args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
