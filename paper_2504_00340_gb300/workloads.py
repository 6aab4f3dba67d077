"""Seeded synthetic workloads for the proton-beam depth march.

Inputs only: grids, beams, densities and default physics constants.  No step
of the method's arithmetic lives here, so both the CUDA library's tests and
benchmark and the CPU oracle may use it.  This module imports nothing else
from the package.

The paper measures against FLUKA on a 4000x80x80 mesh with 500 groups and
20x20 angles (Section 4); no such data is available, so these seeded inputs,
shaped like the paper's pencil beams (Eq. (bdy): Gaussian in y, z, u, v and
E; sigma_u = 1e-6, sigma_E = 1 MeV), stand in for it.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

# Physics constants of the synthetic workloads (MeV, cm, g).  Bragg-Kleeman
# range law R = alpha E^p in water, Highland-type multiple-scattering power,
# and placeholder catastrophic-scatter parameters (the paper fits these to
# FLUKA data and prints no values).
PHYSICS = dict(
    bk_alpha=0.0022,   # cm MeV^-p
    bk_p=1.77,
    x0=36.08,          # radiation length of water, g/cm^2
    mp=938.272,        # proton rest energy, MeV
    es=13.6,           # Highland constant, MeV
    sigma_ct=0.012,    # catastrophic removal cross section, cm^2/g (placeholder)
    lambda_p1=0.05,    # exponential energy transfer rate, 1/MeV (placeholder)
    g_alpha=2.0,       # Gamma angular deflection shape (placeholder)
    g_beta=40.0,       # Gamma angular deflection rate, 1/rad (placeholder)
    s_scale=1.0,
    ts_scale=1.0,
)


@dataclass
class Workload:
    name: str
    ny: int
    nz: int
    nu: int
    nv: int
    ng: int
    e_min: float
    e_max: float
    dy: float = 0.1
    dz: float = 0.1
    dx: float = 0.05
    n_steps: int = 1
    u_max: float = 0.1
    v_max: float = 0.1
    n_scatter: int = 0
    beam: dict = field(default_factory=dict)
    medium: str = "water"
    seed: int = 0
    precision: str = "fp32"
    physics: dict = field(default_factory=lambda: dict(PHYSICS))

    @property
    def na(self) -> int:
        return self.nu * self.nv

    @property
    def e_faces(self) -> np.ndarray:
        return np.linspace(self.e_min, self.e_max, self.ng + 1)

    @property
    def cells_per_step(self) -> int:
        """Phase-space cells (y, z, g, u, v) of one component."""
        return self.ny * self.nz * self.ng * self.na

    @property
    def cell_updates_per_step(self) -> int:
        return self.cells_per_step * (self.n_scatter + 1)

    def grid(self) -> dict:
        return dict(ny=self.ny, nz=self.nz, nu=self.nu, nv=self.nv, dy=self.dy, dz=self.dz,
                    u_max=self.u_max, v_max=self.v_max, e_faces=self.e_faces)

    def density(self, n_steps: int | None = None) -> np.ndarray:
        """rho[s][y][z] in g/cm^3 for depth steps 0..n_steps-1 (cell centred)."""
        n = self.n_steps if n_steps is None else n_steps
        if self.medium == "water":
            return np.ones((n, self.ny, self.nz))
        if self.medium == "slab_phantom":
            return slab_phantom(n, self.ny, self.nz, self.dx, self.dy, self.dz)
        if self.medium == "random_field":
            return random_density(n, self.ny, self.nz, self.dx, self.dy, self.dz, self.seed)
        if self.medium == "random_lateral":
            rng = np.random.default_rng(self.seed)
            return rng.uniform(0.5, 1.5, size=(n, self.ny, self.nz))
        raise ValueError(self.medium)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def slab_phantom(n_steps, ny, nz, dx, dy, dz):
    """Layers along depth: water 0-3 cm, bone (1.85) 3-5 cm, lung (0.26)
    5-10 cm, water beyond; plus a bone cylinder of radius 1 cm whose axis is
    parallel to depth at (y, z) = (2 cm, 0), spanning depths 10-25 cm."""
    x = (np.arange(n_steps) + 0.5) * dx
    y = (np.arange(ny) + 0.5 - ny / 2) * dy
    z = (np.arange(nz) + 0.5 - nz / 2) * dz
    rho = np.ones((n_steps, ny, nz))
    rho[(x >= 3.0) & (x < 5.0)] = 1.85
    rho[(x >= 5.0) & (x < 10.0)] = 0.26
    yy, zz = np.meshgrid(y, z, indexing="ij")
    cyl = (yy - 2.0) ** 2 + zz ** 2 <= 1.0
    for s in np.nonzero((x >= 10.0) & (x < 25.0))[0]:
        rho[s][cyl] = 1.85
    return rho


def random_density(n_steps, ny, nz, dx, dy, dz, seed, corr_len=1.0, mean=1.0, std=0.3, lo=0.2, hi=1.9):
    """Smooth Gaussian random density: white noise filtered by a Gaussian of
    correlation length corr_len (cm) in all three directions, rescaled to the
    given mean and standard deviation, then clipped to [lo, hi]."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((n_steps, ny, nz))
    out = w
    for axis, h in ((0, dx), (1, dy), (2, dz)):
        n = out.shape[axis]
        k = np.fft.fftfreq(n, d=h)
        filt = np.exp(-0.5 * (2 * math.pi * k * corr_len) ** 2)
        shape = [1, 1, 1]
        shape[axis] = n
        out = np.real(np.fft.ifft(np.fft.fft(out, axis=axis) * filt.reshape(shape), axis=axis))
    out = (out - out.mean()) / (out.std() + 1e-300)
    return np.clip(mean + std * out, lo, hi)


def _beam(e0, sigma_lat, sigma_e=1.0, y0=0.0, z0=0.0):
    return dict(e0=e0, sigma_e=sigma_e, y0=y0, z0=z0, sigma_y=sigma_lat, sigma_z=sigma_lat, u0=0.0, v0=0.0,
                sigma_u=1e-6, sigma_v=1e-6)


# The five synthetic workloads.  Sizes follow the single-beam and batched
# configurations the solver is measured on.
WATER100 = Workload(
    name="water100_32x32_g64_a8x8_k1", ny=32, nz=32, nu=8, nv=8, ng=64, e_min=0.0, e_max=110.0,
    dx=0.05, n_steps=180, u_max=0.1, v_max=0.1, n_scatter=1, beam=_beam(100.0, 0.3), precision="fp64")

WATER150 = Workload(
    name="water150_128x128_g256_a16x16", ny=128, nz=128, nu=16, nv=16, ng=256, e_min=0.0, e_max=160.0,
    dx=0.05, n_steps=340, u_max=0.15, v_max=0.15, n_scatter=0, beam=_beam(150.0, 0.4), precision="fp32")

SLAB180 = Workload(
    name="slab180_128x128_g320_a16x16_k1", ny=128, nz=128, nu=16, nv=16, ng=320, e_min=0.0, e_max=200.0,
    dx=0.05, n_steps=500, u_max=0.15, v_max=0.15, n_scatter=1, beam=_beam(180.0, 0.4),
    medium="slab_phantom", precision="mixed")

GRF230 = Workload(
    name="grf230_192x192_g384_a16x16_k3", ny=192, nz=192, nu=16, nv=16, ng=384, e_min=0.0, e_max=240.0,
    dx=0.05, n_steps=660, u_max=0.15, v_max=0.15, n_scatter=3, beam=_beam(230.0, 0.5),
    medium="random_field", seed=20250402, precision="mixed")

# The 100 MeV water beam with the paper's own physics tables (Appendix A:
# Bethe-Bloch with Bragg additivity, screened Rutherford).
WATER100_APPENDIX = WATER100.with_(name="water100_appendix_32x32_g64_a8x8_k1", physics=dict(PHYSICS, model=1))

WORKLOADS = {w.name: w for w in (WATER100, WATER150, SLAB180, GRF230, WATER100_APPENDIX)}


def spot_batch(n_beams=256, seed=20250401, pitch=0.5, sigma_lat=0.3):
    """Batched pencil beams: E0 ~ U(70, 200) MeV, lateral centres on a
    16x16 grid of the given pitch; each beam runs to R(E0) + 1 cm in water
    with ceil(E0 / 0.5 MeV) groups over [0, E0 + 4 sigma_E] and a 64^2 (E0 <=
    135 MeV) or 96^2 lateral grid at 1 mm, 8x8 angles in +-0.1."""
    rng = np.random.default_rng(seed)
    e0 = rng.uniform(70.0, 200.0, size=n_beams)
    side = int(math.ceil(math.sqrt(n_beams)))
    out = []
    for b in range(n_beams):
        iy, iz = divmod(b, side)
        yc = (iy - (side - 1) / 2) * pitch
        zc = (iz - (side - 1) / 2) * pitch
        E0 = float(e0[b])
        rng_cm = PHYSICS["bk_alpha"] * E0 ** PHYSICS["bk_p"]
        n_steps = int(math.ceil((rng_cm + 1.0) / 0.05))
        ng = int(math.ceil(E0 / 0.5))
        lat = 64 if E0 <= 135.0 else 96
        out.append(Workload(
            name=f"spot{b:03d}", ny=lat, nz=lat, nu=8, nv=8, ng=ng, e_min=0.0, e_max=E0 + 4.0,
            dx=0.05, n_steps=n_steps, u_max=0.1, v_max=0.1, n_scatter=0,
            beam=_beam(E0, sigma_lat, y0=0.0, z0=0.0) | {"yc": yc, "zc": zc}, precision="mixed"))
    return out


def random_state(shape, seed, positive=True):
    """Seeded random phase-space state for substep parity tests."""
    rng = np.random.default_rng(seed)
    x = rng.random(shape) if positive else rng.standard_normal(shape)
    return x


def smooth_state(ny, nz, ng, nv, nu, seed):
    """Seeded smooth positive state [g][c][j][i][p][q]: random Gaussian bumps
    in y, z with random amplitudes per (g, c, angle); the slope coefficient
    is kept smaller than the mean so the DG polynomial stays mostly positive."""
    rng = np.random.default_rng(seed)
    y = (np.arange(ny) + 0.5 - ny / 2)
    z = (np.arange(nz) + 0.5 - nz / 2)
    yy, zz = np.meshgrid(y, z, indexing="ij")
    out = np.zeros((ng, 2, nv, nu, ny, nz))
    cy, cz = rng.uniform(-ny / 6, ny / 6), rng.uniform(-nz / 6, nz / 6)
    sy, sz = rng.uniform(ny / 8, ny / 4), rng.uniform(nz / 8, nz / 4)
    bump = np.exp(-0.5 * ((yy - cy) / sy) ** 2 - 0.5 * ((zz - cz) / sz) ** 2)
    amp = rng.random((ng, nv, nu)) + 0.1
    slope = (rng.random((ng, nv, nu)) - 0.5) * 0.6
    out[:, 0] = amp[..., None, None] * bump
    out[:, 1] = (amp * slope)[..., None, None] * bump
    return out
