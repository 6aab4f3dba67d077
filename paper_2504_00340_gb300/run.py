"""Run one named workload through the C ABI and print a short summary.

    python -m paper_2504_00340_gb300.run --workload water150_128x128_g256_a16x16 \
        [--ny 64 --nz 64] [--ng G] [--steps N] [--precision fp32|fp64|mixed] [--autotune] [--vs-fp64]
    python -m paper_2504_00340_gb300.run --spots 256 [--max-gb 48] [--no-graph] [--no-autotune]
    python -m paper_2504_00340_gb300.run --spots 256 --persistent [--no-graph]
    python -m paper_2504_00340_gb300.run --spots-vs-fp64 3

Sizes may be overridden to make reduced cases of the same kernels (e.g. for
profiling).  Prints the per-kernel device times of the march.  --spots runs
the first N spots of the seeded 256-spot batch (bucketed contexts, each
marched as one CUDA graph); under torchrun the buckets are spread over the
ranks and rank 0 prints the totals (device time: max over ranks).
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


def run_spots(a) -> dict:
    import os

    import torch

    from . import spots as S
    from .workloads import spot_batch
    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", 0)))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sp = spot_batch()[:a.spots]
    if a.spot_steps:  # a reduced case of the same spots (profiling): every depth cut to spot_steps
        sp = [w.with_(n_steps=min(w.n_steps, a.spot_steps)) for w in sp]
    if a.persistent:
        if world > 1:
            raise SystemExit("--persistent runs on one GPU")
        t0 = time.perf_counter()
        doses, st = S.run_persistent(sp, use_graph=not a.no_graph, autotune=not a.no_autotune,
                                     max_bytes=int(a.max_gb * (1 << 30)) if a.max_gb_set else None)
        useful = float(st["cell_updates"])
        return {"spots": len(sp), "persistent_launches": st["launches"], "device_ms": st["device_ms"],
                "wall_s": time.perf_counter() - t0, "cell_updates": useful,
                "cell_updates_per_s": useful / (st["device_ms"] * 1e-3), "kernels": st["kernels"],
                "graph": st["graph"], "shapes": st["shapes"],
                "max_dose": float(max(np.abs(d).max() for d in doses.values()))}
    t0 = time.perf_counter()
    doses, st = S.run_shard(sp, rank, world, max_bytes=int(a.max_gb * (1 << 30)), use_graph=not a.no_graph,
                            autotune=not a.no_autotune)
    wall = time.perf_counter() - t0
    dev_ms = st["device_ms"]
    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([dev_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dev_ms = float(t.item())
        n = torch.tensor([st["cell_updates"]], device="cuda", dtype=torch.float64)
        dist.all_reduce(n)
        processed = float(n.item())
        doses = S.gather_doses(doses, rank, world)
    else:
        processed = float(st["cell_updates"])
    out = None
    if rank == 0:
        useful = float(S.useful_cost(sp))
        out = {"spots": len(sp), "ranks": world, "buckets_rank0": st["buckets"], "device_ms": dev_ms,
               "wall_s_rank0": wall, "cell_updates_processed": processed, "cell_updates_useful": useful,
               "cell_updates_per_s": useful / (dev_ms * 1e-3), "kernels_rank0": st["kernels"],
               "tuning_rank0": st["tuning"], "graph": not a.no_graph,
               "max_dose": float(max(np.abs(d).max() for d in doses.values()))}
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def spots_vs_fp64(binding, n):
    """Dose and fluence error of the mixed-precision march against its FP64
    form for n spots of the seeded batch (lowest, highest and evenly spaced
    energies in between), each alone on its own full grid and depth."""
    from .workloads import spot_batch
    sp = sorted(spot_batch(), key=lambda w: w.beam["e0"])
    pick = sorted({round(i * (len(sp) - 1) / max(1, n - 1)) for i in range(n)})
    rows = []
    for i in pick:
        w = sp[i]
        beam = {k: v for k, v in w.beam.items() if k not in ("yc", "zc")}
        w = w.with_(beam=beam)
        mixed, dose, flu = march(binding, w, w.n_steps, "mixed", profile=False)
        ref, dose64, flu64 = march(binding, w, w.n_steps, "fp64", profile=False)
        rows.append({"spot": w.name, "e0": round(w.beam["e0"], 3), "lateral": w.ny, "groups": w.ng,
                     "steps": w.n_steps, "mixed_cell_updates_per_s": mixed["cell_updates_per_s"],
                     "fp64_cell_updates_per_s": ref["cell_updates_per_s"],
                     "dose_err_vs_fp64": float(np.abs(dose - dose64).max() / np.abs(dose64).max()),
                     "fluence_err_vs_fp64": float(np.abs(flu - flu64).max() / np.abs(flu64).max())})
    return rows


def main(argv=None):
    from . import binding
    from .workloads import WORKLOADS
    p = argparse.ArgumentParser()
    p.add_argument("--workload", default="water150_128x128_g256_a16x16", choices=sorted(WORKLOADS))
    p.add_argument("--ny", type=int)
    p.add_argument("--nz", type=int)
    p.add_argument("--ng", type=int)
    p.add_argument("--steps", type=int)
    p.add_argument("--precision", choices=["fp64", "fp32", "mixed"])
    p.add_argument("--straggling", type=float, default=0.0,
                   help="energy straggling: multiple of the Appendix A.2 coefficient (0: off)")
    p.add_argument("--physics-model", type=int, choices=[0, 1],
                   help="0: Bragg-Kleeman + Highland, 1: the paper's Appendix A tables")
    p.add_argument("--energy-form", type=int, choices=[0, 1], help="FP32 energy kernel form (default: tuned)")
    p.add_argument("--angular-form", type=int, choices=range(8), help="angular kernel form (default: tuned)")
    p.add_argument("--energy-angles", type=int, choices=[4, 8, 16], help="angles per energy block")
    p.add_argument("--transport-cols", type=int, choices=[4, 6, 8], help="transport columns per lane")
    p.add_argument("--transport-ctas", type=int, help="resident transport CTAs per SM (0: as many as fit)")
    p.add_argument("--source-form", type=int, choices=(0, 1, 2),
                   help="BF16 source contraction: 0 tile by tile, 1 pipelined, 2 pipelined with swizzled R tiles")
    p.add_argument("--transport", choices=["heun", "cn"], default="heun",
                   help="transport integrator: explicit trapezoid (default) or CN with the slope lagged")
    p.add_argument("--straggling-integrator", choices=["explicit", "cn"], default="explicit",
                   help="straggling inside the CN energy step explicitly (default) or in the CN step")
    p.add_argument("--spots", type=int, default=0, help="run the first N spots of the 256-spot batch")
    p.add_argument("--max-gb", type=float, default=None,
                   help="device workspace per spot bucket (GiB, default 48), or per persistent launch "
                        "(default: the free device memory)")
    p.add_argument("--spot-steps", type=int, default=0, help="cut every spot's depth to this many steps")
    p.add_argument("--persistent", action="store_true",
                   help="--spots through the persistent batch launch (each spot on its own grid)")
    p.add_argument("--no-graph", action="store_true")
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--autotune", action="store_true", help="autotune launch shapes before a workload march")
    p.add_argument("--no-profile", action="store_true", help="no per-kernel event pairs in the timed march")
    p.add_argument("--vs-fp64", action="store_true",
                   help="also march the same workload in FP64 and report the dose and fluence error against it")
    p.add_argument("--spots-vs-fp64", type=int, default=0,
                   help="mixed vs FP64 dose error of N spots of the batch, each on its own full grid")
    a = p.parse_args(argv)
    a.max_gb_set = a.max_gb is not None
    if a.max_gb is None:
        a.max_gb = 48.0
    if a.spots_vs_fp64:
        import torch
        torch.cuda.set_device(0)
        for row in spots_vs_fp64(binding, a.spots_vs_fp64):
            print(json.dumps(row), flush=True)
        return
    if a.spots:
        out = run_spots(a)
        if out is not None:
            print(json.dumps(out))
        return
    w = WORKLOADS[a.workload]
    kw = {k: getattr(a, k) for k in ("ny", "nz", "ng") if getattr(a, k)}
    if a.ng:
        # keep the group width: the energy range scales with the group count
        kw["e_max"] = w.e_min + (w.e_max - w.e_min) * a.ng / w.ng
    if a.straggling or a.physics_model is not None:
        phys = dict(w.physics, t_scale=a.straggling)
        if a.physics_model is not None:
            phys["model"] = a.physics_model
        kw["physics"] = phys
    w = w.with_(**kw)
    steps = a.steps or w.n_steps
    prec = a.precision or w.precision
    import torch
    torch.cuda.set_device(0)
    out, dose, flu = march(binding, w, steps, prec, autotune=a.autotune, profile=not a.no_profile,
                           energy_form=a.energy_form, transport=a.transport, strag_int=a.straggling_integrator,
                           angular_form=a.angular_form,
                           tuning={k: getattr(a, k)
                                   for k in ("energy_angles", "transport_cols", "transport_ctas", "source_form")
                                   if getattr(a, k) is not None})
    out.update({"workload": w.name, "ny": w.ny, "nz": w.nz, "ng": w.ng, "n_scatter": w.n_scatter,
                "medium": w.medium, "physics_model": w.physics.get("model", 0),
                "straggling": w.physics.get("t_scale", 0.0), "transport": a.transport,
                "straggling_integrator": a.straggling_integrator})
    if a.vs_fp64 and prec != "fp64":
        ref, dose64, flu64 = march(binding, w, steps, "fp64", autotune=False, profile=False, transport=a.transport,
                                   strag_int=a.straggling_integrator)
        out["fp64"] = {"cell_updates_per_s": ref["cell_updates_per_s"],
                       "speedup": out["cell_updates_per_s"] / ref["cell_updates_per_s"],
                       "dose_err_vs_fp64": float(np.abs(dose - dose64).max() / np.abs(dose64).max()),
                       "fluence_err_vs_fp64": float(np.abs(flu - flu64).max() / np.abs(flu64).max())}
    print(json.dumps(out))


def march(binding, w, steps, prec, autotune=False, profile=True, energy_form=None, transport="heun",
          strag_int="explicit", angular_form=None, tuning=None):
    """The whole march of workload w (steps depth steps) in the given
    precision: device time by CUDA events around step + flush on the
    context's stream; per-kernel times when profiling."""
    import torch
    s = binding.Solver(w.grid(), nx=steps, dx=w.dx, n_scatter=w.n_scatter, precision=prec, physics=w.physics)
    try:
        if transport != "heun" or strag_int != "explicit":
            s.set_options(transport_integrator=transport, straggling_integrator=strag_int)
        s.set_material(w.density(steps))
        s.launch_beam(**w.beam)
        if autotune:
            s.autotune(2)
        if energy_form is not None:
            s.set_tuning(energy_form=energy_form)
        if angular_form is not None:
            s.set_tuning(angular_form=angular_form)
        if tuning:
            s.set_tuning(**tuning)
        s.set_profiling(profile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        s.step(steps)
        s.flush()
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        dose, flu = s.read_dose(steps), s.read_fluence(steps + 1)
        out = {"steps": steps, "precision": prec, "device_s": ms / 1e3,
               "cell_updates_per_s": w.cell_updates_per_step * steps / (ms / 1e3),
               "max_dose": float(np.abs(dose).max()), "tuning": s.tuning}
        if profile:
            out["kernels"] = {k: list(v) for k, v in s.profile().items()}
        return out, dose, flu
    finally:
        s.close()

if __name__ == "__main__":
    main()
