"""FP64 CPU oracle of the depth-marching proton-beam solver (arXiv 2504.00340).

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or calls anything here, and nothing here imports the
product library.

The arithmetic lives in ``pbs_oracle.c`` (plain C, double precision); this
module compiles it with gcc and marshals numpy arrays through ctypes.  Arrays
of one component use the logical layout ``[g][c][j][i][p][q]`` (energy group,
DG coefficient, angle v, angle u, lateral y, lateral z).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pbs_oracle.c")
_HDR = os.path.join(_HERE, "pbs_oracle.h")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)


class _Grid(ctypes.Structure):
    _fields_ = [("ny", ctypes.c_int), ("nz", ctypes.c_int), ("ng", ctypes.c_int),
                ("nu", ctypes.c_int), ("nv", ctypes.c_int),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double),
                ("u_max", ctypes.c_double), ("v_max", ctypes.c_double),
                ("e_faces", _D)]


class _Phys(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("bk_alpha", "bk_p", "x0", "mp", "es", "sigma_ct", "lambda_p1",
                 "g_alpha", "g_beta", "s_scale", "ts_scale")] + [("model", ctypes.c_int),
                                                                  ("t_scale", ctypes.c_double)]


class _Beam(ctypes.Structure):
    _fields_ = [(n, ctypes.c_double) for n in
                ("e0", "sigma_e", "y0", "z0", "sigma_y", "sigma_z", "u0", "v0",
                 "sigma_u", "sigma_v")]


class _Opts(ctypes.Structure):
    _fields_ = [("n_scatter", ctypes.c_int), ("scheme", ctypes.c_int),
                ("do_energy", ctypes.c_int), ("do_transport", ctypes.c_int),
                ("do_angular", ctypes.c_int)]


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/_build/liboracle.so (gcc, -O2, OpenMP)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < newest:
        tmp = _OUT + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True, cwd=_HERE)
        os.replace(tmp, _OUT)
    return _OUT


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            lib.orc_create.restype = ctypes.c_void_p
            lib.orc_create.argtypes = [ctypes.POINTER(_Grid), ctypes.POINTER(_Phys)]
            lib.orc_destroy.argtypes = [ctypes.c_void_p]
            lib.orc_get_tables.argtypes = [ctypes.c_void_p] + [_D] * 7
            lib.orc_highland.restype = ctypes.c_double
            lib.orc_highland.argtypes = [ctypes.POINTER(_Phys), ctypes.c_double]
            for fn in ("orc_bethe_water", "orc_scat_power_water", "orc_williams_water"):
                getattr(lib, fn).restype = ctypes.c_double
                getattr(lib, fn).argtypes = [ctypes.POINTER(_Phys), ctypes.c_double]
            for fn in ("orc_bethe_element", "orc_sigma_tr_element"):
                getattr(lib, fn).restype = ctypes.c_double
                getattr(lib, fn).argtypes = [ctypes.POINTER(_Phys), ctypes.c_double, ctypes.c_double,
                                             ctypes.c_double]
            lib.orc_energy_blocks.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _D, _D]
            lib.orc_straggle_blocks.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_double, _D, _D, _D]
            lib.orc_straggle_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, _D]
            lib.orc_set_sigma.argtypes = [ctypes.c_void_p, _D]
            lib.orc_set_straggling_table.argtypes = [ctypes.c_void_p, _D]
            lib.orc_set_straggling_cn.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_get_straggling.argtypes = [ctypes.c_void_p, _D, _D]
            lib.orc_energy_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, _D]
            lib.orc_energy_cn_lane.restype = ctypes.c_double
            lib.orc_energy_cn_lane.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D, _D]
            lib.orc_energy_substep.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, _D, _D, _D, _D]
            lib.orc_source.argtypes = [ctypes.c_void_p, _D, _D, _D]
            lib.orc_transport_substep.argtypes = [ctypes.c_void_p, ctypes.c_double, _D]
            lib.orc_transport_apply.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double, _D, _D,
                                                ctypes.c_int]
            lib.orc_set_transport_cn.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_angular_substep.argtypes = [ctypes.c_void_p, ctypes.c_double, _D, _D]
            lib.orc_set_angular_exact.argtypes = [ctypes.c_void_p, ctypes.c_int]
            lib.orc_init_beam.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Beam), _D]
            lib.orc_march.restype = ctypes.c_int
            lib.orc_march.argtypes = [ctypes.c_void_p, ctypes.POINTER(_Opts), ctypes.POINTER(_Beam), _D,
                                      ctypes.c_int, ctypes.c_double, _D, _D, _D, _D]
            lib.orc_fluence.argtypes = [ctypes.c_void_p, _D, ctypes.c_int, _D]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            _lib = lib
    return _lib


def _ptr(a):
    if a is None:
        return ctypes.cast(None, _D)
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(_D)


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


DEFAULT_PHYS = dict(bk_alpha=0.0022, bk_p=1.77, x0=36.08, mp=938.272, es=13.6, sigma_ct=0.012,
                    lambda_p1=0.05, g_alpha=2.0, g_beta=40.0, s_scale=1.0, ts_scale=1.0, model=0,
                    t_scale=0.0)


def num_threads() -> int:
    return _load().orc_num_threads()


def set_threads(n: int) -> None:
    _load().orc_set_threads(int(n))


def highland(e: float, **phys) -> float:
    p = dict(DEFAULT_PHYS)
    p.update(phys)
    return _load().orc_highland(ctypes.byref(_Phys(**p)), float(e))


def _phys(phys):
    p = dict(DEFAULT_PHYS)
    p.update(phys)
    return ctypes.byref(_Phys(**p))


def bethe_water(e: float, **phys) -> float:
    """Mass stopping power of water (MeV cm^2/g), Bethe-Bloch + Bragg additivity."""
    return _load().orc_bethe_water(_phys(phys), float(e))


def bethe_element(z: float, a: float, e: float, **phys) -> float:
    return _load().orc_bethe_element(_phys(phys), float(z), float(a), float(e))


def sigma_tr_element(z: float, a: float, e: float, **phys) -> float:
    """Screened-Rutherford momentum-transfer cross section per atom (cm^2)."""
    return _load().orc_sigma_tr_element(_phys(phys), float(z), float(a), float(e))


def scat_power_water(e: float, **phys) -> float:
    return _load().orc_scat_power_water(_phys(phys), float(e))


def williams_water(e: float, **phys) -> float:
    """Straggling coefficient of water (MeV^2 cm^2/g), Appendix A.2."""
    return _load().orc_williams_water(_phys(phys), float(e))


class Oracle:
    """One grid + physics context.  ``grid`` keys: ny, nz, nu, nv, dy, dz,
    u_max, v_max, e_faces (ng+1 ascending, MeV).  ``phys`` overrides
    DEFAULT_PHYS."""

    def __init__(self, grid: dict, phys: dict | None = None):
        self.lib = _load()
        self.e_faces = _f64(grid["e_faces"])
        self.ng = len(self.e_faces) - 1
        self.ny, self.nz, self.nu, self.nv = (int(grid[k]) for k in ("ny", "nz", "nu", "nv"))
        self.na = self.nu * self.nv
        self.dy, self.dz = float(grid["dy"]), float(grid["dz"])
        self.u_max, self.v_max = float(grid["u_max"]), float(grid["v_max"])
        self.du = 2.0 * self.u_max / (self.nu + 1)
        self.dv = 2.0 * self.v_max / (self.nv + 1)
        p = dict(DEFAULT_PHYS)
        p.update(phys or {})
        self.phys = p
        self._g = _Grid(self.ny, self.nz, self.ng, self.nu, self.nv, self.dy, self.dz, self.u_max, self.v_max,
                        _ptr(self.e_faces))
        self._p = _Phys(**p)
        self.ctx = self.lib.orc_create(ctypes.byref(self._g), ctypes.byref(self._p))
        if not self.ctx:
            raise MemoryError("orc_create failed")

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx:
            self.lib.orc_destroy(ctx)
            self.ctx = None

    # shapes
    @property
    def comp_shape(self):
        return (self.ng, 2, self.nv, self.nu, self.ny, self.nz)

    @property
    def src_shape(self):
        return (self.ng, self.nv, self.nu, self.ny, self.nz)

    def tables(self) -> dict:
        G, na = self.ng, self.na
        out = dict(s_face=np.zeros(G + 1), ts=np.zeros(G), sig=np.zeros(G), p1=np.zeros((G, G)),
                   p2=np.zeros((G, na, na)), u=np.zeros(self.nu), v=np.zeros(self.nv))
        self.lib.orc_get_tables(self.ctx, *(_ptr(out[k]) for k in ("s_face", "ts", "sig", "p1", "p2", "u", "v")))
        out["e_c"] = 0.5 * (self.e_faces[1:] + self.e_faces[:-1])
        out["de"] = np.diff(self.e_faces)
        return out

    def energy_blocks(self, g: int, rho: float):
        agg, aup = np.zeros((2, 2)), np.zeros((2, 2))
        self.lib.orc_energy_blocks(self.ctx, int(g), float(rho), _ptr(agg), _ptr(aup))
        return agg, aup

    def straggle_blocks(self, g: int, rho: float):
        """(alo, agg, aup) of the interior-penalty straggling operator."""
        alo, agg, aup = np.zeros((2, 2)), np.zeros((2, 2)), np.zeros((2, 2))
        self.lib.orc_straggle_blocks(self.ctx, int(g), float(rho), _ptr(alo), _ptr(agg), _ptr(aup))
        return alo, agg, aup

    def straggle_apply(self, rho: float, x):
        x = _f64(x).reshape(-1)
        out = np.zeros_like(x)
        self.lib.orc_straggle_apply(self.ctx, float(rho), _ptr(x), _ptr(out))
        return out

    def set_sigma(self, sig):
        """Removal cross section of every group (ng values, cm^2/g) in place
        of the constant sigma_ct: group g is removed at sig[g] and the source
        it emits into the next component carries sig[g] (Section 4, the
        emitting group's rate)."""
        s = _f64(sig).reshape(self.ng)
        self.lib.orc_set_sigma(self.ctx, _ptr(s))

    def set_straggling_table(self, t_face=None):
        """Straggling coefficient at the faces (ng+1, MeV^2 cm^2/g); None: off.
        Re-folds the drift T'/2 into the stopping power."""
        t = None if t_face is None else _f64(t_face).reshape(self.ng + 1)
        self.lib.orc_set_straggling_table(self.ctx, _ptr(t))

    def set_straggling_cn(self, full: bool):
        """False (default): straggling explicit inside the CN energy step;
        True: straggling inside the CN step as well (block-tridiagonal)."""
        self.lib.orc_set_straggling_cn(self.ctx, int(bool(full)))

    def straggling(self) -> dict:
        out = dict(t_face=np.zeros(self.ng + 1), s_base=np.zeros(self.ng + 1))
        self.lib.orc_get_straggling(self.ctx, _ptr(out["t_face"]), _ptr(out["s_base"]))
        return out

    def energy_apply(self, rho: float, x):
        x = _f64(x).reshape(-1)
        out = np.zeros_like(x)
        self.lib.orc_energy_apply(self.ctx, float(rho), _ptr(x), _ptr(out))
        return out

    def energy_cn_lane(self, rho: float, h: float, x, src_sum=None):
        """One CN step of one lane; x is [g][c] flattened (2G).  Returns
        (x_new, deposited energy content, same from the operator form)."""
        x = _f64(x).reshape(-1).copy()
        s = None if src_sum is None else _f64(src_sum).reshape(-1)
        w = ctypes.c_double(0.0)
        dep = self.lib.orc_energy_cn_lane(self.ctx, float(rho), float(h), _ptr(x), _ptr(s), ctypes.byref(w))
        return x, dep, w.value

    def energy_substep(self, h: float, rho_yz, psi, src_sum=None):
        psi = _f64(psi).copy()
        assert psi.shape == self.comp_shape
        rho_yz = _f64(rho_yz).reshape(self.ny, self.nz)
        s = None if src_sum is None else _f64(src_sum).reshape(self.src_shape)
        edep, edw = np.zeros((self.ny, self.nz)), np.zeros((self.ny, self.nz))
        self.lib.orc_energy_substep(self.ctx, float(h), _ptr(rho_yz), _ptr(psi), _ptr(s), _ptr(edep), _ptr(edw))
        return psi, edep, edw

    def source(self, rho_yz, prev):
        prev = _f64(prev)
        assert prev.shape == self.comp_shape
        rho_yz = _f64(rho_yz).reshape(self.ny, self.nz)
        out = np.zeros(self.src_shape)
        self.lib.orc_source(self.ctx, _ptr(rho_yz), _ptr(prev), _ptr(out))
        return out

    def transport_substep(self, h: float, psi):
        psi = _f64(psi).copy()
        assert psi.shape == self.comp_shape
        self.lib.orc_transport_substep(self.ctx, float(h), _ptr(psi))
        return psi

    def transport_apply(self, uu: float, vv: float, plane, first_order: bool = False):
        """L(plane) of the limited transport operator (or its first-order
        upwind part) for one [ny][nz] plane moving with angle (uu, vv)."""
        f = _f64(plane).reshape(self.ny, self.nz)
        out = np.zeros_like(f)
        self.lib.orc_transport_apply(self.ctx, float(uu), float(vv), _ptr(f), _ptr(out), int(bool(first_order)))
        return out

    def set_transport_cn(self, cn: bool):
        """Transport time integrator: False = explicit trapezoid (default),
        True = Crank-Nicolson with the slope lagged, solved by an upwind sweep."""
        self.lib.orc_set_transport_cn(self.ctx, int(bool(cn)))

    def set_angular_exact(self, exact: bool):
        """Angular time integrator: False = Crank-Nicolson (default), True =
        the exact exponential of each sine mode."""
        self.lib.orc_set_angular_exact(self.ctx, int(bool(exact)))

    def angular_substep(self, h: float, rho_yz, psi):
        psi = _f64(psi).copy()
        assert psi.shape == self.comp_shape
        rho_yz = _f64(rho_yz).reshape(self.ny, self.nz)
        self.lib.orc_angular_substep(self.ctx, float(h), _ptr(rho_yz), _ptr(psi))
        return psi

    def init_beam(self, beam: dict):
        b = _Beam(**_beam_fields(beam))
        psi = np.zeros(self.comp_shape)
        self.lib.orc_init_beam(self.ctx, ctypes.byref(b), _ptr(psi))
        return psi

    def fluence(self, psi):
        psi = _f64(psi)
        k = psi.size // int(np.prod(self.comp_shape))
        out = np.zeros((self.ny, self.nz))
        self.lib.orc_fluence(self.ctx, _ptr(psi), int(k), _ptr(out))
        return out

    def march(self, rho, n_steps: int, dx: float, beam: dict | None = None, psi=None, n_scatter: int = 0,
              scheme: str = "strang", do_energy=True, do_transport=True, do_angular=True):
        """Depth march.  rho is [n_steps][ny][nz] (g/cm^3).  Returns a dict with
        psi [K+1][g][c][j][i][p][q], dose [s][p][q] (MeV/g per proton, difference
        form), dose_w (operator form) and fluence [s+1][p][q]."""
        K = int(n_scatter)
        rho = _f64(rho).reshape(n_steps, self.ny, self.nz)
        shape = (K + 1,) + self.comp_shape
        if psi is None:
            if beam is None:
                raise ValueError("either beam or psi is required")
            psi_arr = np.zeros(shape)
            b = ctypes.byref(_Beam(**_beam_fields(beam)))
        else:
            psi_arr = _f64(psi).reshape(shape).copy()
            b = ctypes.cast(None, ctypes.POINTER(_Beam))
        o = _Opts(K, 0 if scheme == "strang" else 1, int(bool(do_energy)), int(bool(do_transport)),
                  int(bool(do_angular)))
        dose = np.zeros((n_steps, self.ny, self.nz))
        dose_w = np.zeros((n_steps, self.ny, self.nz))
        flu = np.zeros((n_steps + 1, self.ny, self.nz))
        self.lib.orc_march(self.ctx, ctypes.byref(o), b, _ptr(rho), int(n_steps), float(dx), _ptr(psi_arr),
                           _ptr(dose), _ptr(dose_w), _ptr(flu))
        return dict(psi=psi_arr, dose=dose, dose_w=dose_w, fluence=flu)


def _beam_fields(beam: dict) -> dict:
    d = dict(e0=100.0, sigma_e=1.0, y0=0.0, z0=0.0, sigma_y=0.3, sigma_z=0.3, u0=0.0, v0=0.0,
             sigma_u=1e-6, sigma_v=1e-6)
    for k, v in beam.items():
        if k in d:
            d[k] = float(v)
    return d
