"""Lateral domain decomposition of one pencil beam.

Remark 2 of the paper: the energy and angular subsystems act on every
lateral point (y, z) alone, and only the lateral transport couples
neighbouring cells.  So one beam whose phase-space array outgrows a GPU can be
split along y into parts, each a context holding its own rows plus halo rows
that are copies of its neighbours' rows, refreshed before every transport
substep.  The two stages of the explicit trapezoid each reach two cells
upstream, so four halo rows per interior side make each part's own rows
exactly those of the undivided march.

Two drivers over the C ABI:

* ``Domain``: all parts in this process (one or several devices); the halo
  copies run inside the library (``pbs_domain_step``).
* ``DistributedPart``: one part per ``torch.distributed`` rank; each depth
  step runs stage by stage (``pbs_step_stage``) and between the stages the
  halo rows travel between neighbouring ranks by send/recv, packed and
  unpacked with ``pbs_copy_rows``.

The row split and the exchange plan are plain host logic (``split_rows``,
``halo_plan``, ``exchange_halos``), shared by both drivers and testable
without a GPU.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

HALO = 4  # rows: the reach of the two transport stages


@dataclass(frozen=True)
class PartLayout:
    """Rows y_offset .. y_offset+ny-1 of the grid, the first halo_lo and the
    last halo_hi of them halo rows."""
    y_offset: int
    ny: int
    halo_lo: int
    halo_hi: int

    @property
    def own_start(self) -> int:
        return self.y_offset + self.halo_lo

    @property
    def own_end(self) -> int:
        return self.y_offset + self.ny - self.halo_hi


def split_rows(ny_global: int, n_parts: int, halo: int = HALO) -> list[PartLayout]:
    """Split ny_global rows into n_parts parts of nearly equal own rows (the
    first ny_global % n_parts parts get one more), each with halo rows on its
    interior sides.  Every part must own at least `halo` rows, so that its
    neighbours' halos come from its own rows only."""
    if n_parts < 1 or ny_global < n_parts:
        raise ValueError("need 1 <= n_parts <= ny_global")
    base, extra = divmod(ny_global, n_parts)
    if n_parts > 1 and base < halo:
        raise ValueError(f"each part must own at least {halo} rows")
    out, start = [], 0
    for i in range(n_parts):
        own = base + (1 if i < extra else 0)
        lo = halo if i > 0 else 0
        hi = halo if i + 1 < n_parts else 0
        out.append(PartLayout(start - lo, own + lo + hi, lo, hi))
        start += own
    return out


@dataclass(frozen=True)
class HaloMessage:
    """One side of one exchange: send rows send_first..+n_send-1 of this
    part to `peer`, receive n_recv rows from it into recv_first.. (local
    row indices)."""
    peer: int
    send_first: int
    n_send: int
    recv_first: int
    n_recv: int


def halo_plan(layout: list[PartLayout], rank: int) -> list[HaloMessage]:
    """The messages of part `rank` in one halo exchange: to the part below,
    its own first rows that the lower part's upper halo mirrors; to the part
    above, its own last rows that the upper part's lower halo mirrors."""
    me = layout[rank]
    msgs = []
    if rank > 0:
        below = layout[rank - 1]
        msgs.append(HaloMessage(rank - 1, me.halo_lo, below.halo_hi, 0, me.halo_lo))
    if rank + 1 < len(layout):
        above = layout[rank + 1]
        first_sent = me.ny - me.halo_hi - above.halo_lo
        msgs.append(HaloMessage(rank + 1, first_sent, above.halo_lo, me.ny - me.halo_hi, me.halo_hi))
    return msgs


def exchange_halos(layout, rank, pack, unpack, alloc):
    """One halo exchange of part `rank` over torch.distributed: for each
    neighbour, pack(first, n) gives the rows to send (a tensor), alloc(n)
    a tensor to receive n rows into, unpack(first, n, tensor) stores them.
    Receives are posted first; all transfers are waited for before any
    unpack, so the caller may run the next substep right after."""
    import torch.distributed as dist
    reqs, recvs = [], []
    msgs = halo_plan(layout, rank)
    for m in msgs:
        buf = alloc(m.n_recv)
        reqs.append(dist.irecv(buf, src=m.peer))
        recvs.append((m, buf))
    sends = []
    for m in msgs:
        t = pack(m.send_first, m.n_send)
        sends.append(t)  # keep alive until the send completes
        reqs.append(dist.isend(t, dst=m.peer))
    for r in reqs:
        r.wait()
    for m, buf in recvs:
        unpack(m.recv_first, m.n_recv, buf)


def assemble_rows(layout: list[PartLayout], arrays, axis: int = -2) -> np.ndarray:
    """The whole grid's array from the parts' arrays (rows along `axis`),
    each part contributing its own rows."""
    pieces = []
    for lay, a in zip(layout, arrays):
        idx = [slice(None)] * a.ndim
        idx[axis] = slice(lay.halo_lo, lay.ny - lay.halo_hi)
        pieces.append(a[tuple(idx)])
    return np.concatenate(pieces, axis=axis)


class Domain:
    """One beam split along y into n_parts lateral parts held in this
    process, marched in lock-step by the library (pbs_domain_step).
    devices: one CUDA device index per part (default: the current device)."""

    def __init__(self, grid: dict, nx: int, dx: float, n_parts: int, n_scatter: int = 0, precision: str = "fp32",
                 physics: dict | None = None, halo: int = HALO, devices=None):
        import torch

        from .binding import Solver
        self.grid = dict(grid)
        self.ny_global = int(grid["ny"])
        self.layout = split_rows(self.ny_global, n_parts, halo)
        self.devices = list(devices) if devices is not None else [torch.cuda.current_device()] * n_parts
        self.parts = []
        here = torch.cuda.current_device()
        try:
            for lay, dev in zip(self.layout, self.devices):
                torch.cuda.set_device(dev)
                s = Solver(dict(grid, ny=lay.ny), nx=nx, dx=dx, n_scatter=n_scatter, precision=precision,
                           physics=physics, stream=torch.cuda.current_stream(dev))
                s.set_lateral_part(lay.y_offset, self.ny_global, lay.halo_lo, lay.halo_hi)
                self.parts.append(s)
        finally:
            torch.cuda.set_device(here)

    def _each(self, fn):
        import torch
        here = torch.cuda.current_device()
        out = []
        try:
            for s, lay, dev in zip(self.parts, self.layout, self.devices):
                torch.cuda.set_device(dev)
                out.append(fn(s, lay))
            return out
        finally:
            torch.cuda.set_device(here)

    def set_material(self, rho):
        rho = np.asarray(rho, dtype=np.float64)
        self._each(lambda s, lay: s.set_material(rho[:, lay.y_offset:lay.y_offset + lay.ny]))

    def launch_beam(self, **beam):
        self._each(lambda s, lay: s.launch_beam(**beam))

    def set_tables(self, *args, **kw):
        self._each(lambda s, lay: s.set_tables(*args, **kw))

    def step(self, n: int):
        from .binding import pbs_domain_step
        pbs_domain_step([s.ctx for s in self.parts], n)

    def read_dose(self, n_slabs: int | None = None):
        return assemble_rows(self.layout, self._each(lambda s, lay: s.read_dose(n_slabs)))

    def read_fluence(self, n_planes: int | None = None):
        return assemble_rows(self.layout, self._each(lambda s, lay: s.read_fluence(n_planes)))

    def read_psi(self, k: int = 0):
        return assemble_rows(self.layout, self._each(lambda s, lay: s.read_psi(k)))

    def close(self):
        for s in self.parts:
            s.close()
        self.parts = []


class DistributedPart:
    """Part `rank` of one beam split along y over `world` ranks (one GPU
    each, torch.distributed initialised by the caller).  step() runs each
    depth step stage by stage and exchanges halo rows with the neighbouring
    ranks before both transport stages."""

    def __init__(self, grid: dict, nx: int, dx: float, rank: int, world: int, n_scatter: int = 0,
                 precision: str = "fp32", physics: dict | None = None, halo: int = HALO):
        import torch

        from .binding import Solver
        self.rank, self.world = rank, world
        self.layout = split_rows(int(grid["ny"]), world, halo)
        self.me = self.layout[rank]
        self.solver = Solver(dict(grid, ny=self.me.ny), nx=nx, dx=dx, n_scatter=n_scatter, precision=precision,
                             physics=physics)
        self.solver.set_lateral_part(self.me.y_offset, int(grid["ny"]), self.me.halo_lo, self.me.halo_hi)
        self.dtype = torch.float64 if precision == "fp64" else torch.float32
        self.torch = torch

    def set_material(self, rho_global):
        rho = np.asarray(rho_global, dtype=np.float64)
        self.solver.set_material(rho[:, self.me.y_offset:self.me.y_offset + self.me.ny])

    def launch_beam(self, **beam):
        self.solver.launch_beam(**beam)

    def _alloc(self, n):
        s = self.solver
        return self.torch.empty(s.n_planes * n * s.nz, dtype=self.dtype, device="cuda")

    def _pack(self, first, n):
        buf = self._alloc(n)
        self.solver.copy_rows(first, n, True, buf)
        return buf

    def _unpack(self, first, n, buf):
        self.solver.copy_rows(first, n, False, buf)

    def step(self, n: int):
        s = self.solver
        for _ in range(n):
            s.step_stage(0)
            exchange_halos(self.layout, self.rank, self._pack, self._unpack, self._alloc)
            s.step_stage(1)
            s.step_stage(2)
            exchange_halos(self.layout, self.rank, self._pack, self._unpack, self._alloc)
            s.step_stage(3)

    def read_dose_own(self, n_slabs: int | None = None):
        """Dose of this part's own rows [s][own rows][z]."""
        d = self.solver.read_dose(n_slabs)
        return d[:, self.me.halo_lo:self.me.ny - self.me.halo_hi]

    def close(self):
        self.solver.close()
