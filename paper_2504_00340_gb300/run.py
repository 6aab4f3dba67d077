"""Run one named workload through the C ABI and print a short summary.

    python -m paper_2504_00340_gb300.run --workload water150_128x128_g256_a16x16 \
        [--ny 64 --nz 64] [--ng G] [--steps N] [--precision fp32|fp64|mixed]

Sizes may be overridden to make reduced cases of the same kernels (e.g. for
profiling).  Prints the per-kernel device times of the march.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np


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
    a = p.parse_args(argv)
    w = WORKLOADS[a.workload]
    kw = {k: getattr(a, k) for k in ("ny", "nz", "ng") if getattr(a, k)}
    if a.ng:
        # keep the group width: the energy range scales with the group count
        kw["e_max"] = w.e_min + (w.e_max - w.e_min) * a.ng / w.ng
    w = w.with_(**kw)
    steps = a.steps or w.n_steps
    prec = a.precision or w.precision
    import torch
    torch.cuda.set_device(0)
    s = binding.Solver(w.grid(), nx=steps, dx=w.dx, n_scatter=w.n_scatter, precision=prec)
    s.set_material(w.density(steps))
    s.launch_beam(**w.beam)
    s.set_profiling(True)
    t0 = time.perf_counter()
    s.step(steps)
    dose = s.read_dose(steps)
    t = time.perf_counter() - t0
    prof = s.profile()
    out = {"workload": w.name, "ny": w.ny, "nz": w.nz, "ng": w.ng, "steps": steps, "precision": prec,
           "wall_s": t, "cell_updates_per_s": w.cell_updates_per_step * steps / t,
           "max_dose": float(np.abs(dose).max()), "kernels": {k: list(v) for k, v in prof.items()}}
    print(json.dumps(out))
    s.close()


if __name__ == "__main__":
    main()
