"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle
on the same seeded inputs.  Tolerances: FP64 GPU within 1e-10 of the
oracle (relative to the largest value); FP32 within the bounds stated per
test; mixed precision within 1e-3 of the maximum dose."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.workloads import WATER100, random_state, smooth_state

pytestmark = pytest.mark.gpu


def _grid(ny, nz, nu, nv, ng, e_min=0.0, e_max=60.0, dy=0.1, dz=0.1, u_max=0.15):
    return dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=dy, dz=dz, u_max=u_max, v_max=u_max,
                e_faces=np.linspace(e_min, e_max, ng + 1))


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _pair(orc, grid, nx, dx, K, precision, rho=None, seed=0):
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=K, precision=precision)
    o = orc.Oracle(grid)
    if rho is None:
        rho = np.random.default_rng(seed).uniform(0.3, 1.9, size=(nx, grid["ny"], grid["nz"]))
    s.set_material(rho)
    return s, o, rho


def test_tables_match_oracle(orc):
    grid = _grid(4, 4, 6, 4, 40, e_min=0.0, e_max=110.0)
    s = binding.Solver(grid, nx=1, dx=0.05, n_scatter=1, precision="fp64")
    t = s.tables()
    r = orc.Oracle(grid).tables()
    for k in ("s_face", "ts", "sig", "p1", "p2", "u", "v"):
        assert _relerr(t[k], r[k]) < 1e-13, k
    s.close()


def test_appendix_physics_tables_and_march_match_oracle(orc):
    """The paper's own physics (model 1: Bethe-Bloch with Bragg additivity,
    screened Rutherford) built by the library equals the oracle's tables, and
    the K = 1 FP64 march on them equals the oracle's march."""
    grid = _grid(10, 12, 8, 8, 30, e_max=60.0)
    phys = dict(model=1)
    o = orc.Oracle(grid, phys)
    nx, dx = 6, 0.05
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64", physics=phys)
    got, ref = s.tables(), o.tables()
    for k in ("s_face", "ts", "sig", "p1", "p2"):
        assert _relerr(got[k], ref[k]) < 1e-13, k
    rho = np.random.default_rng(12).uniform(0.5, 1.5, size=(nx, 10, 12))
    s.set_material(rho)
    beam = dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)
    s.launch_beam(**beam)
    s.step(nx)
    m = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), m["dose"]) < 1e-10
    assert _relerr(s.read_fluence(), m["fluence"]) < 1e-10
    s.close()


def test_caller_tables_match_oracle(orc):
    """Tables handed in through pbs_set_tables (the oracle's, for other
    physics parameters than the context's) drive the march exactly like the
    built-in ones: tables and the K = 1 march agree with the oracle."""
    grid = _grid(12, 10, 8, 8, 24)
    phys = dict(s_scale=1.2, ts_scale=0.7, sigma_ct=0.02, lambda_p1=0.08)
    o = orc.Oracle(grid, phys)
    t = o.tables()
    nx, dx = 6, 0.05
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    s.set_tables(t["s_face"], t["ts"], t["sig"], phys["lambda_p1"], t["p2"])
    got = s.tables()
    for k in ("s_face", "ts", "sig", "p1", "p2"):
        assert _relerr(got[k], t[k]) < 1e-13, k
    rho = np.random.default_rng(9).uniform(0.5, 1.5, size=(nx, 12, 10))
    s.set_material(rho)
    beam = dict(e0=45.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)
    s.launch_beam(**beam)
    s.step(nx)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < 1e-10
    with pytest.raises(binding.PbsError):
        s.set_tables(t["s_face"], t["ts"], t["sig"], -1.0)
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("ny,nz", [(6, 7), (5, 9)])
def test_energy_substep_with_source_chain(orc, precision, tol, ny, nz):
    """nyz = 42 (even: the packed FP32 form) and 45 (odd: one lane per
    thread), 37 groups, components 0..2 chained by their sources."""
    grid = _grid(ny, nz, 4, 4, 37)
    K = 2
    s, o, rho = _pair(orc, grid, 3, 0.05, K, precision)
    states = [smooth_state(ny, nz, 37, 4, 4, seed=10 + k) for k in range(K + 1)]
    for k in range(K + 1):
        s.write_psi(k, states[k])
    h, slab = 0.025, 1
    s.substep_energy(h, slab, fluence_plane=2)
    # oracle: components in order, source of k from k-1 at start and end (trapezoid)
    ref = [x.copy() for x in states]
    edep = np.zeros((ny, nz))
    src_sum = None
    for k in range(K + 1):
        src_a = o.source(rho[slab], ref[k]) if k < K else None
        ref[k], e, _ = o.energy_substep(h, rho[slab], ref[k], src_sum)
        edep += e
        if k < K:
            src_sum = src_a + o.source(rho[slab], ref[k])
    for k in range(K + 1):
        assert _relerr(s.read_psi(k), ref[k]) < tol, k
    dose = s.read_dose(3)[slab]
    dose_ref = edep / (rho[slab] * 0.05 * 0.1 * 0.1)
    assert _relerr(dose, dose_ref) < 10 * tol
    s.close()
    # the fluence plane receives the particle count of the new state of every component
    s2, _, _ = _pair(orc, grid, 3, 0.05, K, precision)
    for k in range(K + 1):
        s2.write_psi(k, states[k])
    s2.substep_energy(h, slab, fluence_plane=0)
    flu_ref = sum(o.fluence(ref[k]) for k in range(K + 1))
    assert _relerr(s2.read_fluence(1)[0], flu_ref) < 10 * tol
    s2.close()


@pytest.mark.parametrize("cols", [0, 4, 6, 8])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("ny,nz", [(21, 12), (9, 5), (40, 32), (24, 128), (13, 100), (7, 144), (3, 64),
                                   (5, 150), (6, 192), (3, 260), (4, 96), (5, 198)])
def test_transport_substep(orc, precision, tol, ny, nz, cols):
    """Rows of every width class: one lane group, several groups per warp,
    segments with halo lanes, ragged (non-vector) rows; 4 or 6 columns per
    lane (0: chosen by the row width; rows that are not a multiple of the
    lane width take the per-column path)."""
    grid = _grid(ny, nz, 4, 6, 3)
    s, o, _ = _pair(orc, grid, 1, 0.05, 0, precision)
    s.set_tuning(transport_cols=cols)
    psi = random_state((3, 2, 6, 4, ny, nz), seed=ny * nz)
    s.write_psi(0, psi)
    s.substep_transport(0.37)
    ref = o.transport_substep(0.37, psi)
    assert _relerr(s.read_psi(0), ref) < tol
    s.close()


@pytest.mark.parametrize("form", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("nu,nv", [(8, 8), (16, 16), (4, 6)])
def test_angular_substep(orc, precision, tol, nu, nv, form):
    """Packed forms 2 (one slab stack per CTA), 3 (64 registers) and 4 (two
    stacks per CTA); FP64 and the odd lateral count take the direct form."""
    grid = _grid(5, 9, nu, nv, 3)  # nyz = 45: ragged against the 32/16-point tiles
    s, o, rho = _pair(orc, grid, 2, 0.05, 1, precision)
    s.set_tuning(angular_form=form)
    psi = [random_state((3, 2, nv, nu, 5, 9), seed=7 + k) for k in range(2)]
    for k in range(2):
        s.write_psi(k, psi[k])
    s.substep_angular(3.0, 1)
    for k in range(2):
        ref = o.angular_substep(3.0, rho[1], psi[k])
        assert _relerr(s.read_psi(k), ref) < tol
    s.close()


@pytest.mark.parametrize("form", [0, 1, 2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("nu,nv", [(16, 16), (8, 8)])
def test_angular_exact_integrator(orc, precision, tol, form, nu, nv):
    """The exact-exponential angular integrator in every kernel form (direct,
    TMA-staged, packed) against the oracle's."""
    grid = _grid(12, 16, nu, nv, 5)
    s, o, rho = _pair(orc, grid, 2, 0.05, 1, precision)
    s.set_options("exact")
    s.set_tuning(angular_form=form)
    o.set_angular_exact(True)
    psi = [random_state((5, 2, nv, nu, 12, 16), seed=27 + k) for k in range(2)]
    for k in range(2):
        s.write_psi(k, psi[k])
    s.substep_angular(3.0, 1)
    for k in range(2):
        assert _relerr(s.read_psi(k), o.angular_substep(3.0, rho[1], psi[k])) < tol
    s.close()


@pytest.mark.parametrize("nu,nv", [(16, 16), (8, 8), (4, 6), (10, 10)])
def test_angular_packed_forms_agree_bit_for_bit(orc, nu, nv):
    """The packed forms 2-7 (coefficients from the constant bank, or from
    registers in 5-7: the same FP32 magnitudes, zero entries skipped) give the
    same FP32 result, and it matches the oracle; even lateral count 12 x 16,
    three groups (form 4 and 7 take two stacks per CTA: a ragged last pair)."""
    grid = _grid(12, 16, nu, nv, 3)
    s, o, rho = _pair(orc, grid, 2, 0.05, 1, "fp32")
    psi = [random_state((3, 2, nv, nu, 12, 16), seed=41 + k) for k in range(2)]
    out = {}
    for form in (2, 3, 4, 5, 6, 7):
        s.set_tuning(angular_form=form)
        for k in range(2):
            s.write_psi(k, psi[k])
        s.substep_angular(3.0, 1)
        out[form] = [s.read_psi(k) for k in range(2)]
    for form in (3, 4, 5, 6, 7):
        for k in range(2):
            assert np.array_equal(out[form][k], out[2][k]), (form, k)
    for k in range(2):
        assert _relerr(out[5][k], o.angular_substep(3.0, rho[1], psi[k])) < 5e-6
    s.close()


def test_full_march_exact_angular_fp64(orc):
    grid = _grid(14, 12, 8, 8, 24)
    nx, dx = 8, 0.05
    s, o, rho = _pair(orc, grid, nx, dx, 1, "fp64")
    s.set_options("exact")
    o.set_angular_exact(True)
    beam = dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.25)
    s.launch_beam(**beam)
    s.step(nx)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < 1e-10
    o.set_angular_exact(False)
    cn = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(cn["dose"], ref["dose"]) > 1e-9  # the option changes the result
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("ny,nz,nu,nv,ng", [(12, 16, 16, 16, 80), (6, 12, 8, 8, 150), (10, 10, 4, 6, 200)])
def test_angular_substep_tma_pipeline(orc, precision, tol, ny, nz, nu, nv, ng):
    """The TMA-staged persistent form: row pitch a multiple of 16 bytes, a
    ragged last lateral tile (72 or 100 points) or full tiles (192), and
    enough tiles per CTA (two components x 2 ng stacks) that every buffer is
    reused and every barrier phase flips."""
    grid = _grid(ny, nz, nu, nv, ng)
    s, o, rho = _pair(orc, grid, 2, 0.05, 1, precision)
    psi = [random_state((ng, 2, nv, nu, ny, nz), seed=17 + k) for k in range(2)]
    for k in range(2):
        s.write_psi(k, psi[k])
    s.substep_angular(3.0, 1)
    for k in range(2):
        ref = o.angular_substep(3.0, rho[1], psi[k])
        assert _relerr(s.read_psi(k), ref) < tol
    s.close()


@pytest.mark.parametrize("precision,tol,ny,nz,nu,nv", [
    ("fp64", 1e-12, 9, 8, 8, 8), ("fp32", 1e-6, 9, 8, 8, 8), ("mixed", 8e-3, 9, 8, 8, 8),
    # tensor-core path: na = 256 and 128, lateral 72 points (one full and one ragged 64-point tile)
    ("mixed", 8e-3, 9, 8, 16, 16), ("mixed", 8e-3, 8, 9, 8, 16), ("mixed", 8e-3, 20, 16, 16, 16),
    # na = 256 with nyz % 8 != 0: the CUDA-core fallback
    ("mixed", 8e-3, 9, 7, 16, 16)])
def test_source_contraction(orc, precision, tol, ny, nz, nu, nv):
    grid = _grid(ny, nz, nu, nv, 20)
    s, o, rho = _pair(orc, grid, 1, 0.05, 1, precision)
    psi = smooth_state(ny, nz, 20, nv, nu, seed=3)
    s.write_psi(0, psi)
    got = s.eval_source(0, 0)
    ref = o.source(rho[0], psi)
    assert _relerr(got, ref) < tol
    s.close()


@pytest.mark.parametrize("form", [0, 1, 2])
@pytest.mark.parametrize("ny,nz,nu,nv,ng", [(24, 24, 16, 16, 40), (16, 20, 8, 16, 60), (12, 12, 16, 16, 7),
                                             (10, 12, 16, 16, 30)])
def test_source_contraction_tensor_core_forms(orc, form, ny, nz, nu, nv, ng):
    """The tile-by-tile, the pipelined and the pipelined-swizzled tcgen05
    contraction (source_form 0 / 1 / 2) on many groups per CTA (P^2 reloads at group boundaries, every R stage
    and both TMEM accumulators reused) and a ragged last N tile, against the
    oracle in BF16 tolerance."""
    grid = _grid(ny, nz, nu, nv, ng)
    s, o, rho = _pair(orc, grid, 1, 0.05, 1, "mixed")
    s.set_tuning(source_form=form)
    psi = smooth_state(ny, nz, ng, nv, nu, seed=4)
    s.write_psi(0, psi)
    got = s.eval_source(0, 0)
    ref = o.source(rho[0], psi)
    assert _relerr(got, ref) < 8e-3
    s.close()


def test_source_contraction_pipelined_forms_equal_tile_by_tile_on_many_tiles():
    """About ten 64-point tiles per CTA, so that every one of the pipelined
    form's four TMEM accumulators and three R stages is reused several times
    and each CTA crosses group boundaries (P^2 released by an MMA commit and
    reloaded): the pipelined forms issue the same MMAs in the same K order as
    the tile-by-tile form, so their BF16 sources equal it bit for bit."""
    ny = nz = 24
    ng = 160
    grid = _grid(ny, nz, 16, 16, ng)
    s = binding.Solver(grid, nx=1, dx=0.05, n_scatter=1, precision="mixed")
    s.set_material(np.random.default_rng(9).uniform(0.5, 1.5, size=(1, ny, nz)))
    s.write_psi(0, smooth_state(ny, nz, ng, 16, 16, seed=11))
    out = {}
    for form in (0, 1, 2):
        s.set_tuning(source_form=form)
        out[form] = s.eval_source(0, 0)
    assert np.abs(out[0]).max() > 0
    assert np.array_equal(out[1], out[0])
    assert np.array_equal(out[2], out[0])
    s.close()


def test_full_march_fp64(orc):
    grid = _grid(18, 14, 8, 8, 24, e_max=60.0)
    nx, dx = 12, 0.05
    s, o, rho = _pair(orc, grid, nx, dx, 1, "fp64")
    beam = dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.25, y0=0.05)
    s.launch_beam(**beam)
    s.step(5)
    s.step(nx - 5)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < 1e-10
    assert _relerr(s.read_fluence(), ref["fluence"]) < 1e-10
    for k in range(2):
        assert _relerr(s.read_psi(k), ref["psi"][k]) < 1e-10
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp32", 1e-4), ("mixed", 1e-3)])
def test_full_march_reduced_precision(orc, precision, tol):
    grid = _grid(16, 16, 8, 8, 48, e_max=60.0)
    nx, dx = 60, 0.05
    s, o, rho = _pair(orc, grid, nx, dx, 1, precision, rho=np.ones((60, 16, 16)))
    beam = dict(e0=45.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)
    s.launch_beam(**beam)
    s.step(nx)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    d, dr = s.read_dose(), ref["dose"]
    assert np.abs(d - dr).max() / np.abs(dr).max() < tol
    f, fr = s.read_fluence(), ref["fluence"]
    assert np.abs(f - fr).max() / np.abs(fr).max() < tol
    s.close()


def test_full_march_mixed_tensor_core_source(orc):
    """Mixed precision with the BF16 tensor-core source contraction (16x16
    angles, K = 2) against the FP64 oracle: dose within 1e-3 of the maximum."""
    grid = _grid(8, 8, 16, 16, 24, e_max=60.0)
    nx, dx = 16, 0.05
    s, o, rho = _pair(orc, grid, nx, dx, 2, "mixed", rho=np.ones((16, 8, 8)))
    beam = dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)
    s.launch_beam(**beam)
    s.step(nx)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=2)
    d, dr = s.read_dose(), ref["dose"]
    assert np.abs(d - dr).max() / np.abs(dr).max() < 1e-3
    p1, r1 = s.read_psi(1), ref["psi"][1]
    assert np.abs(p1 - r1).max() / np.abs(r1).max() < 1e-2
    s.close()


@pytest.mark.slow
def test_small_workload_full_size_fp64(orc):
    """The 100 MeV / 32x32 / 64 groups / 8x8 angles / primary + 1 workload,
    all 180 steps, FP64 on the GPU against the oracle."""
    w = WATER100
    grid = w.grid()
    rho = w.density()
    s = binding.Solver(grid, nx=w.n_steps, dx=w.dx, n_scatter=w.n_scatter, precision="fp64")
    s.set_material(rho)
    s.launch_beam(**w.beam)
    s.step(w.n_steps)
    ref = orc.Oracle(grid).march(rho, w.n_steps, w.dx, beam=w.beam, n_scatter=w.n_scatter)
    assert _relerr(s.read_dose(), ref["dose"]) < 1e-10
    assert _relerr(s.read_fluence(), ref["fluence"]) < 1e-10
    s.close()
