"""Thin Python binding of the C ABI in include/pbs.h (argument marshalling only).

Every function named ``pbs_*`` here calls the C function of the same name in
``_lib/libpbs.so``; all arithmetic of the method runs in that library's CUDA
kernels.  PyTorch is used only to allocate the caller-owned device workspace
and to name the CUDA stream.  If the library has not been built, or no CUDA
device is present, these calls raise: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build as _build

_lock = threading.Lock()
_lib = None

PBS_FP64, PBS_FP32, PBS_MIXED = 0, 1, 2
PRECISIONS = {"fp64": PBS_FP64, "fp32": PBS_FP32, "mixed": PBS_MIXED}
STATUS = {0: "PBS_OK", -1: "PBS_ERR_ARG", -2: "PBS_ERR_CUDA", -3: "PBS_ERR_NOMEM", -4: "PBS_ERR_STATE",
          -5: "PBS_ERR_TIMEOUT", -6: "PBS_ERR_UNSUPPORTED"}

_D = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


class PbsGrid(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ng", ctypes.c_int), ("nu", ctypes.c_int),
                ("nv", ctypes.c_int), ("nx", ctypes.c_int), ("n_scatter", ctypes.c_int), ("n_beams", ctypes.c_int),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("dx", ctypes.c_double),
                ("u_max", ctypes.c_double), ("v_max", ctypes.c_double), ("e_faces", _D)]


class PbsPhysics(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("bk_alpha", "bk_p", "x0", "mp", "es", "sigma_ct", "lambda_p1",
                                               "g_alpha", "g_beta", "s_scale", "ts_scale")] + [
        ("model", ctypes.c_int), ("t_scale", ctypes.c_double)]


class PbsBeam(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in ("e0", "sigma_e", "y0", "z0", "sigma_y", "sigma_z", "u0", "v0",
                                               "sigma_u", "sigma_v")]


class PbsTuning(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("energy_angles", "energy_form", "transport_ctas", "transport_cols",
                                            "angular_form", "source_form")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class PbsOptions(ctypes.Structure):
    _fields_ = [("angular_integrator", ctypes.c_int), ("transport_integrator", ctypes.c_int),
                ("straggling_integrator", ctypes.c_int)]


class PbsBatchOptions(ctypes.Structure):
    _fields_ = [("use_graph", ctypes.c_int), ("wait_limit_ms", ctypes.c_double), ("hold_beam", ctypes.c_int),
                ("shape", ctypes.c_int), ("transport_cols", ctypes.c_int), ("pipeline", ctypes.c_int)]


class PbsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# (name, restype, argtypes) of every exported entry point of include/pbs.h
SIGNATURES = [
    ("pbs_create", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.POINTER(PbsGrid), ctypes.c_int, _VP]),
    ("pbs_workspace_size", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("pbs_bind_workspace", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("pbs_set_physics", ctypes.c_int, [_VP, ctypes.POINTER(PbsPhysics)]),
    ("pbs_set_tables", ctypes.c_int, [_VP, _D, _D, _D, ctypes.c_double, _D]),
    ("pbs_get_tables", ctypes.c_int, [_VP, _D, _D, _D, _D, _D, _D, _D]),
    ("pbs_set_straggling", ctypes.c_int, [_VP, _D]),
    ("pbs_get_straggling", ctypes.c_int, [_VP, _D, _D]),
    ("pbs_set_material", ctypes.c_int, [_VP, _D, ctypes.c_int]),
    ("pbs_launch_beam", ctypes.c_int, [_VP, ctypes.POINTER(PbsBeam)]),
    ("pbs_launch_beams", ctypes.c_int, [_VP, ctypes.POINTER(PbsBeam), ctypes.c_int]),
    ("pbs_set_beam_steps", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    ("pbs_run", ctypes.c_int, [_VP, ctypes.c_int]),
    ("pbs_autotune", ctypes.c_int, [_VP, ctypes.c_int]),
    ("pbs_set_options", ctypes.c_int, [_VP, ctypes.POINTER(PbsOptions)]),
    ("pbs_get_options", ctypes.c_int, [_VP, ctypes.POINTER(PbsOptions)]),
    ("pbs_set_tuning", ctypes.c_int, [_VP, ctypes.POINTER(PbsTuning)]),
    ("pbs_get_tuning", ctypes.c_int, [_VP, ctypes.POINTER(PbsTuning)]),
    ("pbs_step", ctypes.c_int, [_VP, ctypes.c_int]),
    ("pbs_flush", ctypes.c_int, [_VP]),
    ("pbs_step_stage", ctypes.c_int, [_VP, ctypes.c_int]),
    ("pbs_set_lateral_part", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    ("pbs_domain_step", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.c_int]),
    ("pbs_copy_rows", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, _VP]),
    ("pbs_batch_workspace_size", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    ("pbs_run_batch", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.c_size_t,
                                     ctypes.POINTER(PbsBatchOptions)]),
    ("pbs_batch_autotune", ctypes.c_int, [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.c_size_t, ctypes.c_int,
                                          ctypes.POINTER(PbsBatchOptions)]),
    ("pbs_get_depth", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_int)]),
    ("pbs_checkpoint_size", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_size_t)]),
    ("pbs_checkpoint_save", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("pbs_checkpoint_load", ctypes.c_int, [_VP, _VP, ctypes.c_size_t]),
    ("pbs_read_dose", ctypes.c_int, [_VP, _D, ctypes.c_size_t]),
    ("pbs_read_fluence", ctypes.c_int, [_VP, _D, ctypes.c_size_t]),
    ("pbs_read_psi", ctypes.c_int, [_VP, ctypes.c_int, _D, ctypes.c_size_t]),
    ("pbs_write_psi", ctypes.c_int, [_VP, ctypes.c_int, _D, ctypes.c_size_t]),
    ("pbs_substep_energy", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int, ctypes.c_int]),
    ("pbs_substep_transport", ctypes.c_int, [_VP, ctypes.c_double]),
    ("pbs_substep_angular", ctypes.c_int, [_VP, ctypes.c_double, ctypes.c_int]),
    ("pbs_eval_source", ctypes.c_int, [_VP, ctypes.c_int, ctypes.c_int, _D, ctypes.c_size_t]),
    ("pbs_eval_source_noalloc", ctypes.c_int, [_VP, _VP, _VP, _D, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                               ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, ctypes.c_double, _VP, _VP]),
    ("pbs_kernel_launches", ctypes.c_int, [_VP, ctypes.POINTER(ctypes.c_longlong)]),
    ("pbs_set_profiling", ctypes.c_int, [_VP, ctypes.c_int]),
    ("pbs_profile_read", ctypes.c_int, [_VP, ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                        ctypes.POINTER(ctypes.c_double)]),
    ("pbs_last_error", ctypes.c_char_p, [_VP]),
    ("pbs_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("pbs_destroy", None, [_VP]),
]


def library_path() -> str:
    return _build.LIB


def load_library(build_if_missing: bool = False) -> ctypes.CDLL:
    """Load libpbs.so (building it first if asked).  Raises if it is absent."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if build_if_missing:
                path = _build.build()
            if not os.path.exists(path):
                raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
            lib = ctypes.CDLL(path)
            for name, res, args in SIGNATURES:
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.cast(None, _D)
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_D)


def _check(ctx, status):
    if status != 0:
        lib = load_library()
        msg = lib.pbs_last_error(ctx).decode() if ctx else lib.pbs_status_string(status).decode()
        raise PbsError(status, msg)


# ---------------------------------------------------------------- C-ABI names

def pbs_create(grid: PbsGrid, precision: int, stream: int | None) -> int:
    lib = load_library()
    out = _VP()
    st = lib.pbs_create(ctypes.byref(out), ctypes.byref(grid), int(precision), _VP(stream or 0))
    if st != 0:
        raise PbsError(st, lib.pbs_status_string(st).decode())
    return out.value


def pbs_workspace_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, load_library().pbs_workspace_size(_VP(ctx), ctypes.byref(n)))
    return n.value


def pbs_bind_workspace(ctx, dev_ptr: int, nbytes: int) -> None:
    _check(ctx, load_library().pbs_bind_workspace(_VP(ctx), _VP(dev_ptr), nbytes))


def pbs_set_physics(ctx, phys: PbsPhysics) -> None:
    _check(ctx, load_library().pbs_set_physics(_VP(ctx), ctypes.byref(phys)))


def pbs_set_tables(ctx, s_face, ts, sig_ct, lambda_p1: float, p2=None) -> None:
    _check(ctx, load_library().pbs_set_tables(_VP(ctx), _ptr(s_face), _ptr(ts), _ptr(sig_ct), float(lambda_p1),
                                              _ptr(p2)))


def pbs_get_tables(ctx, s_face, ts, sig, p1, p2, u, v) -> None:
    _check(ctx, load_library().pbs_get_tables(_VP(ctx), *(_ptr(x) for x in (s_face, ts, sig, p1, p2, u, v))))


def pbs_set_straggling(ctx, t_face) -> None:
    _check(ctx, load_library().pbs_set_straggling(_VP(ctx), _ptr(t_face)))


def pbs_get_straggling(ctx, t_face, s_base) -> None:
    _check(ctx, load_library().pbs_get_straggling(_VP(ctx), _ptr(t_face), _ptr(s_base)))


def pbs_set_material(ctx, rho: np.ndarray, n_slabs: int) -> None:
    _check(ctx, load_library().pbs_set_material(_VP(ctx), _ptr(rho), int(n_slabs)))


def pbs_launch_beam(ctx, beam: PbsBeam) -> None:
    _check(ctx, load_library().pbs_launch_beam(_VP(ctx), ctypes.byref(beam)))


def pbs_launch_beams(ctx, beams) -> None:
    arr = (PbsBeam * len(beams))(*beams)
    _check(ctx, load_library().pbs_launch_beams(_VP(ctx), arr, len(beams)))


def pbs_set_beam_steps(ctx, steps) -> None:
    arr = (ctypes.c_int * len(steps))(*[int(x) for x in steps])
    _check(ctx, load_library().pbs_set_beam_steps(_VP(ctx), arr, len(steps)))


def pbs_run(ctx, use_graph: bool) -> None:
    _check(ctx, load_library().pbs_run(_VP(ctx), int(bool(use_graph))))


def pbs_autotune(ctx, reps: int = 3) -> None:
    _check(ctx, load_library().pbs_autotune(_VP(ctx), int(reps)))


def pbs_set_options(ctx, options: PbsOptions) -> None:
    _check(ctx, load_library().pbs_set_options(_VP(ctx), ctypes.byref(options)))


def pbs_get_options(ctx) -> PbsOptions:
    o = PbsOptions()
    _check(ctx, load_library().pbs_get_options(_VP(ctx), ctypes.byref(o)))
    return o


def pbs_set_tuning(ctx, tuning: PbsTuning) -> None:
    _check(ctx, load_library().pbs_set_tuning(_VP(ctx), ctypes.byref(tuning)))


def pbs_get_tuning(ctx) -> PbsTuning:
    t = PbsTuning()
    _check(ctx, load_library().pbs_get_tuning(_VP(ctx), ctypes.byref(t)))
    return t


def pbs_step(ctx, n_steps: int) -> None:
    _check(ctx, load_library().pbs_step(_VP(ctx), int(n_steps)))


def pbs_flush(ctx) -> None:
    _check(ctx, load_library().pbs_flush(_VP(ctx)))


def pbs_step_stage(ctx, stage: int) -> None:
    _check(ctx, load_library().pbs_step_stage(_VP(ctx), int(stage)))


def pbs_set_lateral_part(ctx, y_offset: int, ny_global: int, halo_lo: int, halo_hi: int) -> None:
    _check(ctx, load_library().pbs_set_lateral_part(_VP(ctx), int(y_offset), int(ny_global), int(halo_lo),
                                                    int(halo_hi)))


def pbs_domain_step(ctxs, n_steps: int) -> None:
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    _check(ctxs[0], load_library().pbs_domain_step(arr, len(ctxs), int(n_steps)))


def pbs_copy_rows(ctx, first_row: int, n_rows: int, to_buffer: bool, dev_ptr: int) -> None:
    _check(ctx, load_library().pbs_copy_rows(_VP(ctx), int(first_row), int(n_rows), int(bool(to_buffer)),
                                             _VP(dev_ptr)))


def pbs_batch_workspace_size(ctxs) -> int:
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    n = ctypes.c_size_t()
    _check(ctxs[0], load_library().pbs_batch_workspace_size(arr, len(ctxs), ctypes.byref(n)))
    return n.value


def pbs_run_batch(ctxs, dev_ptr: int, nbytes: int, use_graph: bool = False, wait_limit_ms: float = 0.0,
                  hold_beam: int = -1, shape: int = 0, transport_cols: int = 0, pipeline: int = 0) -> None:
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    opts = PbsBatchOptions(int(bool(use_graph)), float(wait_limit_ms), int(hold_beam), int(shape),
                           int(transport_cols), int(pipeline))
    _check(ctxs[0], load_library().pbs_run_batch(arr, len(ctxs), _VP(dev_ptr), nbytes, ctypes.byref(opts)))


def pbs_batch_autotune(ctxs, dev_ptr: int, nbytes: int, steps: int = 6) -> dict:
    """The batch shape and transport columns the autotuner picks (see
    pbs_batch_autotune); the beams restart from their projections."""
    arr = (_VP * len(ctxs))(*[_VP(c) for c in ctxs])
    opts = PbsBatchOptions(0, 0.0, -1, 0, 0, 0)
    _check(ctxs[0], load_library().pbs_batch_autotune(arr, len(ctxs), _VP(dev_ptr), nbytes, int(steps),
                                                      ctypes.byref(opts)))
    return {"shape": opts.shape, "transport_cols": opts.transport_cols, "pipeline": opts.pipeline}


def pbs_checkpoint_size(ctx) -> int:
    n = ctypes.c_size_t()
    _check(ctx, load_library().pbs_checkpoint_size(_VP(ctx), ctypes.byref(n)))
    return n.value


def pbs_checkpoint_save(ctx, buf: np.ndarray) -> None:
    assert buf.dtype == np.uint8 and buf.flags["C_CONTIGUOUS"]
    _check(ctx, load_library().pbs_checkpoint_save(_VP(ctx), _VP(buf.ctypes.data), buf.size))


def pbs_checkpoint_load(ctx, buf: np.ndarray) -> None:
    assert buf.dtype == np.uint8 and buf.flags["C_CONTIGUOUS"]
    _check(ctx, load_library().pbs_checkpoint_load(_VP(ctx), _VP(buf.ctypes.data), buf.size))


def pbs_get_depth(ctx) -> int:
    s = ctypes.c_int()
    _check(ctx, load_library().pbs_get_depth(_VP(ctx), ctypes.byref(s)))
    return s.value


def pbs_read_dose(ctx, out: np.ndarray) -> None:
    _check(ctx, load_library().pbs_read_dose(_VP(ctx), _ptr(out), out.size))


def pbs_read_fluence(ctx, out: np.ndarray) -> None:
    _check(ctx, load_library().pbs_read_fluence(_VP(ctx), _ptr(out), out.size))


def pbs_read_psi(ctx, k: int, out: np.ndarray) -> None:
    _check(ctx, load_library().pbs_read_psi(_VP(ctx), int(k), _ptr(out), out.size))


def pbs_write_psi(ctx, k: int, arr: np.ndarray) -> None:
    _check(ctx, load_library().pbs_write_psi(_VP(ctx), int(k), _ptr(arr), arr.size))


def pbs_substep_energy(ctx, h: float, slab: int, fluence_plane: int = -1) -> None:
    _check(ctx, load_library().pbs_substep_energy(_VP(ctx), float(h), int(slab), int(fluence_plane)))


def pbs_substep_transport(ctx, h: float) -> None:
    _check(ctx, load_library().pbs_substep_transport(_VP(ctx), float(h)))


def pbs_substep_angular(ctx, h: float, slab: int) -> None:
    _check(ctx, load_library().pbs_substep_angular(_VP(ctx), float(h), int(slab)))


def pbs_eval_source(ctx, k_from: int, slab: int, out: np.ndarray) -> None:
    _check(ctx, load_library().pbs_eval_source(_VP(ctx), int(k_from), int(slab), _ptr(out), out.size))


def pbs_eval_source_noalloc(psi_k_ptr: int, rho_ptr: int, p2_ptr: int, e_faces: np.ndarray, ng: int, nu: int,
                            nv: int, ny: int, nz: int, u_max: float, v_max: float, sigma_ct: float,
                            lambda_p1: float, src_ptr: int, stream: int | None) -> None:
    """Allocation-free source evaluation on caller-owned FP32 device buffers
    (raw device pointers); see include/pbs.h."""
    ef = np.ascontiguousarray(np.asarray(e_faces, dtype=np.float64))
    st = load_library().pbs_eval_source_noalloc(_VP(psi_k_ptr), _VP(rho_ptr), _VP(p2_ptr), _ptr(ef), int(ng), int(nu),
                                                int(nv), int(ny), int(nz), float(u_max), float(v_max),
                                                float(sigma_ct), float(lambda_p1), _VP(src_ptr), _VP(stream or 0))
    if st != 0:
        raise PbsError(st, load_library().pbs_status_string(st).decode())


def pbs_kernel_launches(ctx) -> int:
    n = ctypes.c_longlong()
    _check(ctx, load_library().pbs_kernel_launches(_VP(ctx), ctypes.byref(n)))
    return n.value


KERNEL_KINDS = {"energy": 0, "transport": 1, "angular": 2, "source": 3, "queue": 4}


def pbs_set_profiling(ctx, on: bool) -> None:
    _check(ctx, load_library().pbs_set_profiling(_VP(ctx), int(bool(on))))


def pbs_profile_read(ctx, kind: int):
    n, ms = ctypes.c_longlong(), ctypes.c_double()
    _check(ctx, load_library().pbs_profile_read(_VP(ctx), int(kind), ctypes.byref(n), ctypes.byref(ms)))
    return n.value, ms.value


def pbs_last_error(ctx) -> str:
    return load_library().pbs_last_error(_VP(ctx)).decode()


def pbs_destroy(ctx) -> None:
    if ctx:
        load_library().pbs_destroy(_VP(ctx))


# ---------------------------------------------------------------- convenience

DEFAULT_PHYSICS = dict(bk_alpha=0.0022, bk_p=1.77, x0=36.08, mp=938.272, es=13.6, sigma_ct=0.012, lambda_p1=0.05,
                       g_alpha=2.0, g_beta=40.0, s_scale=1.0, ts_scale=1.0, model=0, t_scale=0.0)
_BEAM_DEFAULTS = dict(e0=100.0, sigma_e=1.0, y0=0.0, z0=0.0, sigma_y=0.3, sigma_z=0.3, u0=0.0, v0=0.0,
                      sigma_u=1e-6, sigma_v=1e-6)


def _batch_workspace(solvers, workspace):
    import torch
    nbytes = pbs_batch_workspace_size([s.ctx for s in solvers])
    if workspace is None or workspace.numel() < nbytes:
        workspace = torch.empty(max(nbytes, 256), dtype=torch.uint8, device="cuda")
    return workspace


def run_batch(solvers, use_graph: bool = False, wait_limit_ms: float = 0.0, hold_beam: int = -1, workspace=None,
              shape: int = 0, transport_cols: int = 0, pipeline: int = 0):
    """March every Solver of the list (one beam each, see pbs_run_batch) in
    one persistent launch on their common stream.  The batch workspace is a
    torch tensor allocated here unless given (keep it alive while the batch
    runs: it is returned)."""
    workspace = _batch_workspace(solvers, workspace)
    pbs_run_batch([s.ctx for s in solvers], workspace.data_ptr(), workspace.numel(), use_graph, wait_limit_ms,
                  hold_beam, shape, transport_cols, pipeline)
    return workspace


def autotune_batch(solvers, steps: int = 6, workspace=None):
    """(options picked by pbs_batch_autotune, workspace)."""
    workspace = _batch_workspace(solvers, workspace)
    return pbs_batch_autotune([s.ctx for s in solvers], workspace.data_ptr(), workspace.numel(), steps), workspace


class Solver:
    """One context on the current CUDA device, holding n_beams beams on one grid.

    grid: dict with ny, nz, nu, nv, dy, dz, u_max, v_max, e_faces (ng+1, MeV);
    nx: number of depth steps (dose slabs); dx: step (cm); n_scatter: K;
    precision: 'fp64' | 'fp32' | 'mixed'; stream: a torch.cuda.Stream or None
    (the current stream).  With n_beams > 1, read_dose / read_fluence return
    arrays with a leading beam axis and component k of read_psi is component
    k % (K+1) of beam k // (K+1)."""

    def __init__(self, grid: dict, nx: int, dx: float, n_scatter: int = 0, precision: str = "fp32",
                 stream=None, physics: dict | None = None, n_beams: int = 1):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required (the library has no CPU path)")
        self.torch = torch
        self.e_faces = np.ascontiguousarray(np.asarray(grid["e_faces"], dtype=np.float64))
        self.ny, self.nz, self.nu, self.nv = (int(grid[k]) for k in ("ny", "nz", "nu", "nv"))
        self.ng = len(self.e_faces) - 1
        self.na = self.nu * self.nv
        self.nx, self.dx, self.K = int(nx), float(dx), int(n_scatter)
        self.n_beams = int(n_beams)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._g = PbsGrid(self.ny, self.nz, self.ng, self.nu, self.nv, self.nx, self.K, self.n_beams, float(grid["dy"]),
                          float(grid["dz"]), self.dx, float(grid["u_max"]), float(grid["v_max"]),
                          _ptr(self.e_faces))
        self._precision = PRECISIONS[precision]
        self.ctx = pbs_create(self._g, self._precision, self.stream.cuda_stream)
        nbytes = pbs_workspace_size(self.ctx)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        pbs_bind_workspace(self.ctx, self.workspace.data_ptr(), nbytes)
        self.set_physics(**(physics or {}))

    def close(self):
        if getattr(self, "ctx", None):
            pbs_destroy(self.ctx)
            self.ctx = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def comp_shape(self):
        return (self.ng, 2, self.nv, self.nu, self.ny, self.nz)

    def set_physics(self, **kw):
        p = dict(DEFAULT_PHYSICS)
        p.update(kw)
        pbs_set_physics(self.ctx, PbsPhysics(**p))

    def set_tables(self, s_face, ts, sig_ct, lambda_p1: float, p2=None):
        """Caller-supplied tables (see pbs_set_tables): s_face[ng+1], ts[ng],
        sig_ct[ng], lambda_p1, optional p2[ng][na][na]."""
        f = lambda x: None if x is None else np.ascontiguousarray(np.asarray(x, dtype=np.float64))  # noqa: E731
        pbs_set_tables(self.ctx, f(s_face), f(ts), f(sig_ct), lambda_p1, f(p2))

    def set_straggling(self, t_face=None):
        """Straggling coefficient at the group faces (ng+1, MeV^2 cm^2/g), or
        None to switch straggling off (see pbs_set_straggling)."""
        t = None if t_face is None else np.ascontiguousarray(np.asarray(t_face, dtype=np.float64))
        if t is not None and t.shape != (self.ng + 1,):
            raise ValueError("t_face must have ng + 1 entries")
        pbs_set_straggling(self.ctx, t)

    def straggling(self) -> dict:
        out = dict(t_face=np.zeros(self.ng + 1), s_base=np.zeros(self.ng + 1))
        pbs_get_straggling(self.ctx, out["t_face"], out["s_base"])
        return out

    def tables(self) -> dict:
        G, na = self.ng, self.na
        out = dict(s_face=np.zeros(G + 1), ts=np.zeros(G), sig=np.zeros(G), p1=np.zeros((G, G)),
                   p2=np.zeros((G, na, na)), u=np.zeros(self.nu), v=np.zeros(self.nv))
        pbs_get_tables(self.ctx, out["s_face"], out["ts"], out["sig"], out["p1"], out["p2"], out["u"], out["v"])
        return out

    def set_material(self, rho):
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64)).reshape(-1, self.ny, self.nz)
        pbs_set_material(self.ctx, rho, rho.shape[0])

    @staticmethod
    def _beam(beam: dict) -> PbsBeam:
        b = dict(_BEAM_DEFAULTS)
        b.update({k: float(v) for k, v in beam.items() if k in b})
        return PbsBeam(**b)

    def launch_beam(self, **beam):
        pbs_launch_beam(self.ctx, self._beam(beam))

    def launch_beams(self, beams):
        """One beam dict per beam of the context."""
        pbs_launch_beams(self.ctx, [self._beam(b) for b in beams])

    def set_lateral_part(self, y_offset: int, ny_global: int, halo_lo: int, halo_hi: int):
        """Declare this context a lateral part of a beam split along y (see
        pbs_set_lateral_part); before launch_beam."""
        pbs_set_lateral_part(self.ctx, y_offset, ny_global, halo_lo, halo_hi)

    def step_stage(self, stage: int):
        """Stage 0..3 of the next depth step (see pbs_step_stage)."""
        pbs_step_stage(self.ctx, stage)

    def copy_rows(self, first_row: int, n_rows: int, to_buffer: bool, buf):
        """Rows of every psi plane to / from a device tensor buf laid out
        [plane][row][z] (see pbs_copy_rows)."""
        pbs_copy_rows(self.ctx, first_row, n_rows, to_buffer, buf.data_ptr())

    @property
    def n_planes(self) -> int:
        """psi planes (ny x nz cells) of all components: the rows of
        copy_rows' buffer per copied row."""
        return self.n_beams * (self.K + 1) * self.ng * 2 * self.na

    def set_beam_steps(self, steps):
        pbs_set_beam_steps(self.ctx, steps)

    def run(self, use_graph: bool = True):
        """The whole march of every beam to its depth (restarting from the
        launched projections), optionally as one CUDA graph launch."""
        pbs_run(self.ctx, use_graph)

    def autotune(self, reps: int = 3):
        pbs_autotune(self.ctx, reps)

    @property
    def tuning(self) -> dict:
        """Launch shapes and kernel forms: energy_angles, energy_form,
        transport_ctas, transport_cols, angular_form, source_form."""
        return pbs_get_tuning(self.ctx).as_dict()

    def set_options(self, angular_integrator: str = "cn", transport_integrator: str = "heun",
                    straggling_integrator: str = "explicit"):
        """Method options: angular_integrator 'cn' (Crank-Nicolson, default)
        or 'exact' (exact exponential of each sine mode); transport_integrator
        'heun' (explicit trapezoid, default) or 'cn' (Crank-Nicolson with the
        slope lagged, upwind sweep); straggling_integrator 'explicit' (inside
        the CN energy step, default) or 'cn' (in the CN step, block
        elimination)."""
        pbs_set_options(self.ctx, PbsOptions({"cn": 0, "exact": 1}[angular_integrator],
                                             {"heun": 0, "cn": 1}[transport_integrator],
                                             {"explicit": 0, "cn": 1}[straggling_integrator]))

    def set_tuning(self, **kw):
        t = pbs_get_tuning(self.ctx)
        for k, v in kw.items():
            setattr(t, k, int(v))
        pbs_set_tuning(self.ctx, t)

    def step(self, n: int):
        pbs_step(self.ctx, n)

    def flush(self):
        pbs_flush(self.ctx)

    def checkpoint(self) -> np.ndarray:
        """The march state as a host byte array (pbs_checkpoint_save)."""
        buf = np.empty(pbs_checkpoint_size(self.ctx), dtype=np.uint8)
        pbs_checkpoint_save(self.ctx, buf)
        return buf

    def restore(self, buf: np.ndarray):
        pbs_checkpoint_load(self.ctx, np.ascontiguousarray(buf, dtype=np.uint8))

    @property
    def depth(self) -> int:
        return pbs_get_depth(self.ctx)

    def read_dose(self, n_slabs: int | None = None):
        n = self.nx if n_slabs is None else n_slabs
        out = np.zeros((self.n_beams, n, self.ny, self.nz))
        pbs_read_dose(self.ctx, out)
        return out[0] if self.n_beams == 1 else out

    def read_fluence(self, n_planes: int | None = None):
        n = self.depth + 1 if n_planes is None else n_planes
        out = np.zeros((self.n_beams, n, self.ny, self.nz))
        pbs_read_fluence(self.ctx, out)
        return out[0] if self.n_beams == 1 else out

    def read_psi(self, k: int = 0):
        out = np.zeros(self.comp_shape)
        pbs_read_psi(self.ctx, k, out)
        return out

    def write_psi(self, k: int, arr):
        a = np.ascontiguousarray(np.asarray(arr, dtype=np.float64)).reshape(self.comp_shape)
        pbs_write_psi(self.ctx, k, a)

    def psi_view(self, k: int = 0):
        """Device view (torch tensor, no copy) of component k in the documented
        layout [g][c][v][u][y][z]; psi sits at the start of the workspace.
        The view bypasses the API: call flush() after step() before reading it."""
        torch = self.torch
        dt = torch.float64 if self._precision == PBS_FP64 else torch.float32
        n = int(np.prod(self.comp_shape))
        esz = 8 if dt == torch.float64 else 4
        raw = self.workspace[k * n * esz:(k + 1) * n * esz]
        return raw.view(dt).view(self.comp_shape)

    def substep_energy(self, h, slab, fluence_plane=-1):
        pbs_substep_energy(self.ctx, h, slab, fluence_plane)

    def substep_transport(self, h):
        pbs_substep_transport(self.ctx, h)

    def substep_angular(self, h, slab):
        pbs_substep_angular(self.ctx, h, slab)

    def eval_source(self, k_from: int, slab: int):
        out = np.zeros((self.ng, self.nv, self.nu, self.ny, self.nz))
        pbs_eval_source(self.ctx, k_from, slab, out)
        return out

    @property
    def kernel_launches(self) -> int:
        return pbs_kernel_launches(self.ctx)

    def set_profiling(self, on: bool):
        pbs_set_profiling(self.ctx, on)

    def profile(self) -> dict:
        """{kind: (launches, total_ms)} of the kernels timed since set_profiling(True)."""
        return {k: pbs_profile_read(self.ctx, v) for k, v in KERNEL_KINDS.items()}
