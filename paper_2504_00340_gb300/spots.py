"""Batched pencil-beam spots: planning (host logic) and execution.

A spot batch is a list of beams, each with its own energy, depth range and
lateral grid.  The solver marches several beams in one context when they
share a grid, so the planner groups the spots into buckets:

  * same lateral/angular grid, depth step, scattering order and precision;
  * one energy grid per bucket, that of its highest-energy spot; a spot joins
    only if its own group count is at least (1 - max_waste) of the bucket's,
    so at most that fraction of its groups is empty work;
  * spots ordered by depth range, longest first (the context's launches then
    cover a shrinking prefix of beams as the shorter ones stop);
  * a bucket's device workspace stays below max_bytes.

Each bucket then runs as one context: launch all beams, optionally autotune
the launch shapes, and march the whole bucket as one recorded CUDA graph.
With several ranks the buckets are spread over them by estimated cost
(longest-processing-time first); ranks exchange nothing but the final doses,
which the caller gathers.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .workloads import Workload


@dataclass
class Bucket:
    """Spots marched together in one context."""
    grid_key: tuple
    ng: int
    e_max: float
    e_min: float
    members: list = field(default_factory=list)  # indices into the spot list, depth-descending
    steps: list = field(default_factory=list)    # depth steps per member (non-increasing)

    @property
    def nx(self) -> int:
        return self.steps[0] if self.steps else 0


def _grid_key(w: Workload) -> tuple:
    return (w.ny, w.nz, w.nu, w.nv, w.dy, w.dz, w.dx, w.u_max, w.v_max, w.n_scatter, w.precision, w.medium)


def workspace_bytes(ny, nz, nu, nv, ng, nx, n_scatter, n_beams, precision) -> int:
    """Device workspace of a context (the library's layout, each region
    rounded up to 256 bytes)."""
    rs = 8 if precision == "fp64" else 4
    ss = {"fp64": 8, "fp32": 4, "mixed": 2}[precision]
    na, nyz = nu * nv, ny * nz
    comp = ng * 2 * na * nyz
    nsrc = ng * na * nyz if n_scatter > 0 else 0
    r256 = lambda x: (x + 255) // 256 * 256  # noqa: E731
    parts = [n_beams * (n_scatter + 1) * comp * rs,
             2 * n_beams * nsrc * ss, 2 * n_beams * nsrc * ss,
             nx * nyz * rs, n_beams * nx * nyz * 8, n_beams * (nx + 1) * nyz * 8,
             ng * 10 * rs, ng * rs, (ng * na * na * ss if n_scatter > 0 else 0),
             n_beams * (2 * ng + na + ny + nz) * 8, 64]
    return sum(r256(p) for p in parts)


def plan_buckets(spots: list[Workload], max_bytes: int = 48 << 30, max_waste: float = 0.1) -> list[Bucket]:
    """Group spots into buckets (see the module docstring).  Deterministic:
    spots are taken in order of decreasing energy, ties by index."""
    order = sorted(range(len(spots)), key=lambda i: (-spots[i].e_max, i))
    open_: dict[tuple, Bucket] = {}
    out: list[Bucket] = []
    for i in order:
        w = spots[i]
        key = _grid_key(w)
        b = open_.get(key)
        if b is not None:
            fits_e = w.ng >= (1.0 - max_waste) * b.ng and w.e_max <= b.e_max
            nx = max([spots[m].n_steps for m in b.members] + [w.n_steps])
            fits_m = workspace_bytes(w.ny, w.nz, w.nu, w.nv, b.ng, nx, w.n_scatter, len(b.members) + 1,
                                     w.precision) <= max_bytes
            if not (fits_e and fits_m):
                b = None
        if b is None:
            if workspace_bytes(w.ny, w.nz, w.nu, w.nv, w.ng, w.n_steps, w.n_scatter, 1, w.precision) > max_bytes:
                raise ValueError(f"spot {w.name} alone needs more than max_bytes")
            b = Bucket(grid_key=key, ng=w.ng, e_max=w.e_max, e_min=w.e_min)
            open_[key] = b
            out.append(b)
        b.members.append(i)
    for b in out:
        b.members.sort(key=lambda i: (-spots[i].n_steps, i))
        b.steps = [spots[i].n_steps for i in b.members]
    return out


def bucket_cost(b: Bucket, spots: list[Workload]) -> int:
    """Phase-space cell-updates the bucket's march performs (every marching
    beam over the bucket's energy grid)."""
    w = spots[b.members[0]]
    return sum(w.ny * w.nz * w.na * b.ng * (w.n_scatter + 1) * s for s in b.steps)


def useful_cost(spots: list[Workload]) -> int:
    """Cell-updates of the spots on their own energy grids."""
    return sum(w.cell_updates_per_step * w.n_steps for w in spots)


def shard_buckets(buckets: list[Bucket], spots: list[Workload], world_size: int) -> list[list[int]]:
    """Assign bucket indices to ranks, longest first to the least-loaded rank
    (ties to the lower rank).  Every bucket goes to exactly one rank."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    load = [0] * world_size
    out: list[list[int]] = [[] for _ in range(world_size)]
    for j in sorted(range(len(buckets)), key=lambda j: (-bucket_cost(buckets[j], spots), j)):
        r = min(range(world_size), key=lambda r: (load[r], r))
        out[r].append(j)
        load[r] += bucket_cost(buckets[j], spots)
    for r in range(world_size):
        out[r].sort()
    return out


def bucket_grid(b: Bucket, spots: list[Workload]) -> dict:
    w = spots[b.members[0]]
    return dict(ny=w.ny, nz=w.nz, nu=w.nu, nv=w.nv, dy=w.dy, dz=w.dz, u_max=w.u_max, v_max=w.v_max,
                e_faces=np.linspace(b.e_min, b.e_max, b.ng + 1))


def run_bucket(b: Bucket, spots: list[Workload], *, use_graph: bool = True, autotune: bool = True):
    """March one bucket on the current CUDA device.  Returns
    ({spot index: dose [steps][ny][nz]}, device time of the march in ms (CUDA
    events around the run call on the context's stream), kernels launched by
    the context, chosen launch shapes)."""
    import torch

    from . import binding
    w0 = spots[b.members[0]]
    s = binding.Solver(bucket_grid(b, spots), nx=b.nx, dx=w0.dx, n_scatter=w0.n_scatter, precision=w0.precision,
                       n_beams=len(b.members), physics=w0.physics)
    try:
        s.set_material(w0.with_(n_steps=b.nx).density())
        s.set_beam_steps(b.steps)
        s.launch_beams([{k: v for k, v in spots[i].beam.items() if k not in ("yc", "zc")} for i in b.members])
        if autotune:
            s.autotune(2)
        if use_graph:
            s.run(True)  # records the graph (and runs once)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        s.run(use_graph)
        e1.record(s.stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        dose = s.read_dose(b.nx)
        if len(b.members) == 1:
            dose = dose[None]
        out = {i: dose[j, :b.steps[j]].copy() for j, i in enumerate(b.members)}
        return out, ms, s.kernel_launches, s.tuning
    finally:
        s.close()


def total_dose(spots: list[Workload], doses: dict, ny: int, nz: int) -> np.ndarray:
    """Sum the spots' doses on a common lateral frame: spot i's grid is centred
    on its centre (yc, zc) (cm), shifted by whole cells onto a frame of ny x nz
    cells of the spots' cell size centred at 0.  Depth axis: the longest spot's."""
    depth = max(d.shape[0] for d in doses.values())
    out = np.zeros((depth, ny, nz))
    for i, d in doses.items():
        w = spots[i]
        oy = int(round(w.beam.get("yc", 0.0) / w.dy)) + (ny - w.ny) // 2
        oz = int(round(w.beam.get("zc", 0.0) / w.dz)) + (nz - w.nz) // 2
        y0, y1 = max(oy, 0), min(oy + w.ny, ny)
        z0, z1 = max(oz, 0), min(oz + w.nz, nz)
        if y0 < y1 and z0 < z1:
            out[:d.shape[0], y0:y1, z0:z1] += d[:, y0 - oy:y1 - oy, z0 - oz:z1 - oz]
    return out


def gather_doses(local: dict, rank: int, world_size: int):
    """Collect every rank's {spot index: dose} on rank 0 through
    torch.distributed (the process group must be initialised; any backend).
    Returns the merged dict, ordered by spot index, on rank 0 and None on the
    other ranks.  A spot reported by two ranks is an error."""
    import torch.distributed as dist
    parts = [None] * world_size if rank == 0 else None
    dist.gather_object(local, parts, dst=0)
    if rank != 0:
        return None
    merged: dict = {}
    for part in parts:
        for k, v in part.items():
            if k in merged:
                raise RuntimeError(f"spot {k} was marched by two ranks")
            merged[k] = v
    return dict(sorted(merged.items()))


def run_shard(spots: list[Workload], rank: int = 0, world_size: int = 1, *, max_bytes: int = 48 << 30,
              use_graph: bool = True, autotune: bool = True, march=None):
    """Plan the batch, march this rank's buckets and return ({spot: dose},
    stats).  `march(bucket, spots)` replaces run_bucket (same return value)
    for host-only tests of the planning and gathering logic."""
    march = march or (lambda b, sp: run_bucket(b, sp, use_graph=use_graph, autotune=autotune))
    buckets = plan_buckets(spots, max_bytes=max_bytes)
    mine = shard_buckets(buckets, spots, world_size)[rank]
    doses: dict = {}
    stats = dict(buckets=len(mine), device_ms=0.0, kernels=0, cell_updates=0, tuning=[])
    for j in mine:
        out, ms, kernels, tuning = march(buckets[j], spots)
        doses.update(out)
        stats["device_ms"] += ms
        stats["kernels"] += kernels
        stats["cell_updates"] += bucket_cost(buckets[j], spots)
        stats["tuning"].append(tuning)
    return doses, stats


def plan_waves(spots: list[Workload], max_bytes: int) -> list[list[int]]:
    """Spots of the persistent batch, longest depth first (they lead every
    round of the device queue), cut into waves whose workspaces fit
    max_bytes together; each wave is one persistent launch (the whole batch
    when it fits)."""
    order = sorted(range(len(spots)), key=lambda i: (-spots[i].n_steps, i))
    waves, cur, used = [], [], 0
    for i in order:
        w = spots[i]
        b = workspace_bytes(w.ny, w.nz, w.nu, w.nv, w.ng, w.n_steps, w.n_scatter, 1, w.precision)
        if b > max_bytes:
            raise ValueError(f"spot {w.name} alone needs more than max_bytes")
        if cur and used + b > max_bytes:
            waves.append(cur)
            cur, used = [], 0
        cur.append(i)
        used += b
    if cur:
        waves.append(cur)
    return waves


def run_persistent(spots: list[Workload], *, max_bytes: int | None = None, use_graph: bool = False,
                   autotune: bool = True):
    """March the spots through the persistent batch (pbs_run_batch): every
    spot its own context on its own grid (its own energy groups, no bucket
    and no empty groups), as few launches as memory allows, with the CTA
    shape the batch autotuner picks on a few depth steps of the wave.
    Returns ({spot: dose [steps][ny][nz]}, stats with the device time of the
    timed launches (CUDA events on the stream))."""
    import torch

    from . import binding
    if max_bytes is None:
        max_bytes = torch.cuda.mem_get_info()[0] - (6 << 30)
    waves = plan_waves(spots, max_bytes)
    doses: dict = {}
    stats = dict(launches=len(waves), device_ms=0.0, kernels=0, cell_updates=useful_cost(spots),
                 graph=use_graph, shapes=[])
    for wave in waves:
        solvers = []
        try:
            for i in wave:
                w = spots[i]
                s = binding.Solver(w.grid(), nx=w.n_steps, dx=w.dx, n_scatter=w.n_scatter, precision=w.precision,
                                   physics=w.physics)
                solvers.append(s)
                s.set_material(w.density())
                s.launch_beam(**{k: v for k, v in w.beam.items() if k not in ("yc", "zc")})
            opts, ws = binding.autotune_batch(solvers, steps=4) if autotune else ({}, None)
            stats["shapes"].append(opts)
            if use_graph:
                ws = binding.run_batch(solvers, use_graph=True, workspace=ws, **opts)  # records the graph
            k0 = sum(s.kernel_launches for s in solvers)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(solvers[0].stream)
            ws = binding.run_batch(solvers, use_graph=use_graph, workspace=ws, **opts)
            e1.record(solvers[0].stream)
            e1.synchronize()
            stats["device_ms"] += e0.elapsed_time(e1)
            stats["kernels"] += sum(s.kernel_launches for s in solvers) - k0
            for s, i in zip(solvers, wave):
                doses[i] = s.read_dose()
        finally:
            for s in solvers:
                s.close()
            torch.cuda.empty_cache()
    return dict(sorted(doses.items())), stats


__all__ = ["Bucket", "plan_buckets", "shard_buckets", "bucket_cost", "useful_cost", "workspace_bytes",
           "bucket_grid", "run_bucket", "total_dose", "gather_doses", "run_shard", "plan_waves", "run_persistent"]
