"""GPU parity of energy straggling (Section 3.2 with T != 0, Appendix A.2)
against the oracle: the tables (Williams coefficient, drift folded into the
stopping power), one energy substep with dose, the fused back-to-back
substeps of the march (the second scan one group behind the first), batched
beams, caller-given coefficients, the graph-recorded march, and the
stability bound of the explicit straggling step.  FP32 runs both kernel
forms: one lane per thread, and the packed FP32x2 form."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.workloads import random_state

pytestmark = pytest.mark.gpu


def _grid(ny, nz, nu, nv, ng, e_max=60.0, d=0.1, u_max=0.15):
    return dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=d, dz=d, u_max=u_max, v_max=u_max,
                e_faces=np.linspace(0.0, e_max, ng + 1))


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


FORMS = [("fp64", 0), ("fp32", 0), ("fp32", 1)]


@pytest.mark.parametrize("phys", [dict(t_scale=1.0), dict(model=1, t_scale=1.0), dict(t_scale=25.0)])
def test_tables_match_oracle(orc, phys):
    grid = _grid(4, 4, 4, 4, 40, e_max=80.0)
    s = binding.Solver(grid, nx=2, dx=0.05, precision="fp64", physics=phys)
    o = orc.Oracle(grid, phys)
    st, ot = s.straggling(), o.straggling()
    assert np.allclose(st["t_face"], ot["t_face"], rtol=1e-13, atol=0)
    assert np.allclose(st["s_base"], ot["s_base"], rtol=1e-13, atol=0)
    assert np.allclose(s.tables()["s_face"], o.tables()["s_face"], rtol=1e-13, atol=0)
    assert st["t_face"].min() > 0.08
    s.close()


@pytest.mark.parametrize("precision,form", FORMS)
@pytest.mark.parametrize("ng,ny,nz", [(37, 6, 10), (64, 3, 33)])
def test_energy_substep_with_straggling(orc, precision, form, ng, ny, nz):
    """One E substep (explicit straggling inside CN): psi and dose (odd
    ny nz takes the one-lane form in FP32 too)."""
    tol = 1e-12 if precision == "fp64" else 3e-6
    phys = dict(t_scale=20.0)  # exaggerated so that the straggling part is well above rounding
    grid = _grid(ny, nz, 4, 4, ng)
    rho = np.random.default_rng(ng).uniform(0.4, 1.9, size=(1, ny, nz))
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision, physics=phys)
    s.set_tuning(energy_form=form)
    s.set_material(rho)
    psi = np.abs(random_state((ng, 2, 4, 4, ny, nz), seed=ng + 1))
    s.write_psi(0, psi)
    s.substep_energy(0.025, 0)
    o = orc.Oracle(grid, phys)
    ref, edep, _ = o.energy_substep(0.025, rho[0], psi)
    assert _relerr(s.read_psi(0), ref) < tol
    dose_ref = edep / (rho[0] * 0.05 * 0.1 * 0.1)
    assert _relerr(s.read_dose(1)[0], dose_ref) < (1e-11 if precision == "fp64" else 2e-5)
    # the straggling term is not negligible here
    plain = orc.Oracle(grid, dict(t_scale=0.0)).energy_substep(0.025, rho[0], psi)[0]
    assert _relerr(plain, ref) > 1e3 * tol
    s.close()


@pytest.mark.parametrize("precision,tol,form", [("fp64", 1e-10, 0), ("fp32", 2e-5, 0), ("fp32", 2e-5, 1),
                                                ("mixed", 1e-3, 1)])
def test_march_with_straggling(orc, precision, tol, form):
    """Full Strang march, K = 1 (fused pairs, source chain), Appendix-A
    physics with straggling: dose and fluence against the oracle."""
    phys = dict(model=1, t_scale=1.0)
    grid = _grid(12, 10, 8, 8, 48, e_max=60.0) if precision != "mixed" else _grid(12, 10, 16, 16, 48, e_max=60.0)
    nx, dx = 9, 0.05
    rho = np.random.default_rng(21).uniform(0.5, 1.6, size=(nx, 12, 10))
    beam = dict(e0=42.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.2, y0=0.05)
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision, physics=phys)
    s.set_tuning(energy_form=form)
    s.set_material(rho)
    s.launch_beam(**beam)
    s.step(4)
    s.step(nx - 4)
    ref = orc.Oracle(grid, phys).march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < tol
    assert _relerr(s.read_fluence(), ref["fluence"]) < tol
    if precision == "fp64":
        assert _relerr(s.read_psi(0), ref["psi"][0]) < 1e-10
        assert _relerr(s.read_psi(1), ref["psi"][1]) < 1e-10
    s.close()


@pytest.mark.parametrize("precision,form", FORMS)
def test_batch_and_graph_with_straggling(orc, precision, form):
    """Two beams with their own depths, straggling on: each equals the
    oracle's single-beam march; the recorded graph gives the same result as
    the launch sequence."""
    phys = dict(t_scale=3.0)
    grid = _grid(10, 12, 8, 8, 30)
    nx, dx = 6, 0.05
    rho = np.random.default_rng(4).uniform(0.6, 1.4, size=(nx, 10, 12))
    beams = [dict(e0=45.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.25), dict(e0=38.0, sigma_e=0.8, sigma_y=0.3, z0=0.1)]
    steps = [6, 4]
    out = []
    for use_graph in (None, True):
        s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision, n_beams=2, physics=phys)
        s.set_tuning(energy_form=form)
        s.set_material(rho)
        s.set_beam_steps(steps)
        s.launch_beams(beams)
        if use_graph is None:
            s.step(nx)
        else:
            s.run(True)
            s.run(True)
        out.append(s.read_dose())
        s.close()
    o = orc.Oracle(grid, phys)
    tol = 1e-10 if precision == "fp64" else 2e-5
    for b, beam in enumerate(beams):
        ref = o.march(rho[:steps[b]], steps[b], dx, beam=beam, n_scatter=1)
        assert _relerr(out[0][b, :steps[b]], ref["dose"]) < tol, b
    assert _relerr(out[1], out[0]) < (1e-12 if precision == "fp64" else 1e-6)


@pytest.mark.parametrize("precision,form", FORMS)
def test_caller_straggling_table(orc, precision, form):
    """pbs_set_straggling with an arbitrary coefficient (rising and falling
    with E) on top of the built-in stopping power; switching it off again
    restores the plain substep."""
    ng = 28
    grid = _grid(5, 8, 4, 4, ng)
    t_face = 0.5 + 0.4 * np.sin(np.linspace(0.0, 5.0, ng + 1)) ** 2
    rho = np.full((1, 5, 8), 1.2)
    psi = np.abs(random_state((ng, 2, 4, 4, 5, 8), seed=2))
    tol = 1e-12 if precision == "fp64" else 3e-6
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision)
    s.set_tuning(energy_form=form)
    s.set_material(rho)
    s.set_straggling(t_face)
    s.write_psi(0, psi)
    s.substep_energy(0.025, 0)
    o = orc.Oracle(grid)
    o.set_straggling_table(t_face)
    assert _relerr(s.read_psi(0), o.energy_substep(0.025, rho[0], psi)[0]) < tol
    s.set_straggling(None)
    s.write_psi(0, psi)
    s.substep_energy(0.025, 0)
    assert _relerr(s.read_psi(0), orc.Oracle(grid).energy_substep(0.025, rho[0], psi)[0]) < tol
    with pytest.raises(binding.PbsError):
        s.set_straggling(-t_face)
    s.close()


def test_unstable_explicit_straggling_is_refused():
    """Fine groups, a thick step and dense material put the explicit
    straggling step beyond its stability bound: the march refuses to start;
    a thinner substep passes."""
    grid = _grid(4, 4, 4, 4, 200, e_max=20.0)  # dE = 0.1 MeV
    s = binding.Solver(grid, nx=2, dx=2.0, precision="fp32", physics=dict(t_scale=1.0))
    s.set_material(np.full((2, 4, 4), 1.9))
    s.launch_beam(e0=15.0, sigma_e=0.5)
    with pytest.raises(binding.PbsError):
        s.step(1)
    with pytest.raises(binding.PbsError):
        s.substep_energy(1.0, 0)
    s.substep_energy(0.002, 0)
    s.close()


# ---- straggling inside the Crank-Nicolson step (block elimination), pbs_options.straggling_integrator = 1

@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 3e-6)])
@pytest.mark.parametrize("ng,ny,nz", [(37, 6, 10), (64, 3, 33)])
def test_energy_substep_full_cn(orc, precision, tol, ng, ny, nz):
    phys = dict(t_scale=20.0)
    grid = _grid(ny, nz, 4, 4, ng)
    rho = np.random.default_rng(ng + 7).uniform(0.4, 1.9, size=(1, ny, nz))
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision, physics=phys)
    s.set_options(straggling_integrator="cn")
    s.set_material(rho)
    psi = np.abs(random_state((ng, 2, 4, 4, ny, nz), seed=ng + 3))
    s.write_psi(0, psi)
    s.substep_energy(0.025, 0, 0)
    o = orc.Oracle(grid, phys)
    o.set_straggling_cn(True)
    ref, edep, _ = o.energy_substep(0.025, rho[0], psi)
    assert _relerr(s.read_psi(0), ref) < tol
    assert _relerr(s.read_dose(1)[0], edep / (rho[0] * 0.05 * 0.1 * 0.1)) < (1e-11 if precision == "fp64" else 2e-5)
    # fluence after the substep: du dv sum_g dE psi^1 summed over the angles
    de = np.diff(grid["e_faces"])
    du = 2 * grid["u_max"] / 5
    flu_ref = du * du * np.einsum("g,gjipq->pq", de, ref[:, 0])
    assert _relerr(s.read_fluence(1)[0], flu_ref) < (1e-12 if precision == "fp64" else 3e-6)
    # and it differs from the explicit form
    expl = orc.Oracle(grid, phys).energy_substep(0.025, rho[0], psi)[0]
    assert _relerr(expl, ref) > 1e3 * tol
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 2e-5), ("mixed", 1e-3)])
def test_march_full_cn(orc, precision, tol):
    """Two beams with their own depths, K = 1, Appendix-A physics: each beam
    against the oracle's full-CN march of that beam alone."""
    phys = dict(model=1, t_scale=1.0)
    grid = _grid(12, 10, 8, 8, 48, e_max=60.0) if precision != "mixed" else _grid(12, 10, 16, 16, 48, e_max=60.0)
    nx, dx = 7, 0.05
    rho = np.random.default_rng(23).uniform(0.5, 1.6, size=(nx, 12, 10))
    beams = [dict(e0=42.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.2, y0=0.05), dict(e0=36.0, sigma_e=0.8, sigma_y=0.3)]
    steps = [7, 5]
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision, physics=phys, n_beams=2)
    s.set_options(straggling_integrator="cn")
    s.set_material(rho)
    s.set_beam_steps(steps)
    s.launch_beams(beams)
    s.step(3)
    s.step(nx - 3)
    dose, flu = s.read_dose(), s.read_fluence()
    o = orc.Oracle(grid, phys)
    o.set_straggling_cn(True)
    for b, beam in enumerate(beams):
        ref = o.march(rho[:steps[b]], steps[b], dx, beam=beam, n_scatter=1)
        assert _relerr(dose[b, :steps[b]], ref["dose"]) < tol, b
        assert _relerr(flu[b, :steps[b] + 1], ref["fluence"]) < tol, b
        if precision == "fp64":
            assert _relerr(s.read_psi(2 * b + 1), ref["psi"][1]) < 1e-10, b
    s.close()


def test_full_cn_has_no_stability_bound(orc):
    """The configuration the explicit form refuses runs in CN and matches the
    oracle's CN substep."""
    grid = _grid(4, 4, 4, 4, 200, e_max=20.0)
    phys = dict(t_scale=1.0)
    s = binding.Solver(grid, nx=2, dx=2.0, precision="fp64", physics=phys)
    s.set_material(np.full((2, 4, 4), 1.9))
    s.set_options(straggling_integrator="cn")
    psi = np.abs(random_state((200, 2, 4, 4, 4, 4), seed=4))
    s.write_psi(0, psi)
    s.substep_energy(1.0, 0)
    o = orc.Oracle(grid, phys)
    o.set_straggling_cn(True)
    assert _relerr(s.read_psi(0), o.energy_substep(1.0, np.full((4, 4), 1.9), psi)[0]) < 1e-11
    s.close()
