"""Degenerate and edge cases of the CUDA path against the oracle: one- and
two-row planes, single-column rows, the smallest angle grid, a single energy
group, vacuum slabs (rho = 0) inside the march, and empty calls."""
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


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("ny,nz", [(1, 8), (2, 12), (4, 1), (1, 1), (2, 3)])
def test_transport_tiny_planes(orc, precision, tol, ny, nz):
    grid = _grid(ny, nz, 4, 4, 2)
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision)
    psi = random_state((2, 2, 4, 4, ny, nz), seed=ny * 31 + nz)
    s.write_psi(0, psi)
    s.substep_transport(0.3)
    ref = orc.Oracle(grid).transport_substep(0.3, psi)
    assert _relerr(s.read_psi(0), ref) < tol
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
def test_angular_smallest_grid(orc, precision, tol):
    grid = _grid(4, 6, 2, 2, 3)
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision)
    s.set_material(np.full((1, 4, 6), 1.3))
    psi = random_state((3, 2, 2, 2, 4, 6), seed=5)
    s.write_psi(0, psi)
    s.substep_angular(2.0, 0)
    ref = orc.Oracle(grid).angular_substep(2.0, np.full((4, 6), 1.3), psi)
    assert _relerr(s.read_psi(0), ref) < tol
    s.close()


def test_single_group_march(orc):
    grid = _grid(8, 8, 4, 4, 1, e_max=20.0)
    nx, dx = 5, 0.05
    rho = np.ones((nx, 8, 8))
    beam = dict(e0=10.0, sigma_e=1.0, sigma_y=0.2, sigma_z=0.2)
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    s.set_material(rho)
    s.launch_beam(**beam)
    s.step(nx)
    ref = orc.Oracle(grid).march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < 1e-10
    assert _relerr(s.read_fluence(), ref["fluence"]) < 1e-10
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_vacuum_gap(orc, precision, tol):
    """Slabs of rho = 0 inside the march: no energy loss, no scattering, no
    dose there; transport continues."""
    grid = _grid(10, 12, 8, 8, 20)
    nx, dx = 8, 0.05
    rho = np.ones((nx, 10, 12))
    rho[2:5] = 0.0
    rho[6, :5] = 0.0  # a half-vacuum slab
    beam = dict(e0=45.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.25)
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision)
    s.set_material(rho)
    s.launch_beam(**beam)
    s.step(nx)
    d = s.read_dose()
    ref = orc.Oracle(grid).march(rho, nx, dx, beam=beam, n_scatter=1)
    assert not d[2:5].any() and not d[6, :5].any()
    assert _relerr(d, ref["dose"]) < tol
    assert _relerr(s.read_fluence(), ref["fluence"]) < tol
    s.close()


def test_empty_calls():
    grid = _grid(6, 6, 4, 4, 8)
    s = binding.Solver(grid, nx=3, dx=0.05, precision="fp32", n_beams=2)
    s.set_material(np.ones((3, 6, 6)))
    s.launch_beams([dict(e0=30.0), dict(e0=20.0)])
    s.step(0)
    assert s.depth == 0
    assert not s.read_dose(3).any()  # no step marched: no dose
    f = s.read_fluence(1)
    assert f.shape == (2, 1, 6, 6) and np.all(f.sum(axis=(1, 2, 3)) > 0)  # the entrance plane of both beams
    s.set_beam_steps([0, 0])
    s.launch_beams([dict(e0=30.0), dict(e0=20.0)])
    s.run(True)  # no beam marches: the graph holds only the restart
    assert s.depth == 0 and not s.read_dose(3).any()
    with pytest.raises(binding.PbsError):
        s.step(4)  # past the material
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_resume(orc, precision):
    """March 3 steps, checkpoint (with the closing half still deferred),
    march 3 more; a fresh context restored from the checkpoint and marched
    the same 3 steps gives the same dose, fluence and psi; both equal the
    oracle's 6-step march (FP64)."""
    grid = _grid(10, 12, 8, 8, 20)
    nx, dx = 6, 0.05
    rho = np.random.default_rng(11).uniform(0.5, 1.5, size=(nx, 10, 12))
    beams = [dict(e0=45.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.25), dict(e0=38.0, sigma_e=1.0, sigma_y=0.3)]

    def make():
        s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision, n_beams=2)
        s.set_material(rho)
        return s

    a = make()
    a.set_beam_steps([6, 5])
    a.launch_beams(beams)
    a.step(3)
    ck = a.checkpoint()
    a.step(3)
    ref = (a.read_dose(), a.read_fluence(), a.read_psi(0), a.read_psi(3))
    b = make()
    b.restore(ck)
    assert b.depth == 3
    b.step(3)
    got = (b.read_dose(), b.read_fluence(), b.read_psi(0), b.read_psi(3))
    for x, y in zip(got, ref):
        assert _relerr(x, y) < (1e-12 if precision == "fp64" else 1e-6)
    if precision == "fp64":
        o = orc.Oracle(grid).march(rho, nx, dx, beam=beams[0], n_scatter=1)
        assert _relerr(got[0][0], o["dose"]) < 1e-10
    bad = ck.copy()
    bad[:8] = 0
    with pytest.raises(binding.PbsError):
        b.restore(bad)
    other = binding.Solver(grid, nx=nx, dx=dx, n_scatter=0, precision=precision, n_beams=2)
    with pytest.raises(binding.PbsError):
        other.restore(ck)  # another scattering order
    for s in (a, b, other):
        s.close()


# byte offsets of fields in the checkpoint header: magic[8], then 4-byte ints
# version, precision, ny, nz, ng, nu, nv, nx, K, B, steps_done, pending,
# have_beam, n_slabs_at_save, angular, transport, straggling integrators, pad,
# then the 8-byte table and material hashes
_CK_STEPS, _CK_PENDING, _CK_HAVE_BEAM, _CK_ANGULAR = 48, 52, 56, 64


def _put_int(buf, off, v):
    out = buf.copy()
    out[off:off + 4] = np.frombuffer(np.int32(v).tobytes(), dtype=np.uint8)
    return out


def test_checkpoint_rejects_inconsistent_headers():
    """A checkpoint whose header cannot describe a marched state, or that was
    marched with other options, tables or density, is refused before any
    device work; the context stays usable and a good checkpoint still
    restores."""
    grid = _grid(6, 8, 4, 4, 12)
    nx, dx = 4, 0.05
    rho = np.random.default_rng(2).uniform(0.5, 1.5, size=(nx, 6, 8))
    a = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    a.set_material(rho)
    a.launch_beam(e0=40.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.25)
    a.step(2)
    ck = a.checkpoint()  # pending closing half of step 1
    assert int(np.frombuffer(ck[_CK_PENDING:_CK_PENDING + 4].tobytes(), dtype=np.int32)[0]) == 1
    b = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    b.set_material(rho)
    bad = [
        _put_int(_put_int(ck, _CK_STEPS, 0), _CK_PENDING, 1),   # deferred half with no marched step
        _put_int(ck, _CK_PENDING, 2),                           # flag out of range
        _put_int(ck, _CK_HAVE_BEAM, 7),
        _put_int(ck, _CK_STEPS, nx + 1),                        # depth beyond the grid
        _put_int(ck, _CK_STEPS, -1),
        _put_int(ck, _CK_ANGULAR, 1),                           # marched with the exact angular integrator
    ]
    for i, buf in enumerate(bad):
        with pytest.raises(binding.PbsError):
            b.restore(buf)
        assert b.depth == 0, i
    # another density field
    c = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    c.set_material(rho * 1.01)
    with pytest.raises(binding.PbsError):
        c.restore(ck)
    # other options on the restoring side
    b.set_options(angular_integrator="exact")
    with pytest.raises(binding.PbsError):
        b.restore(ck)
    b.set_options(angular_integrator="cn")
    # other tables (a different removal cross section)
    t = a.tables()
    d = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64")
    d.set_tables(t["s_face"], t["ts"], t["sig"] * 2.0, 0.05, t["p2"])
    d.set_material(rho)
    with pytest.raises(binding.PbsError):
        d.restore(ck)
    # the good one restores and continues like the original
    b.restore(ck)
    assert b.depth == 2
    a.step(2)
    b.step(2)
    assert _relerr(b.read_dose(), a.read_dose()) < 1e-12
    for s in (a, b, c, d):
        s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
def test_maximum_group_count(orc, precision, tol):
    """ng = 2048, the largest group count the library accepts: the group table
    no longer fits the packed energy kernel's shared memory, so the one-lane
    form runs; one E substep with dose against the oracle."""
    ng = 2048
    grid = _grid(4, 6, 2, 2, ng, e_max=300.0)
    s = binding.Solver(grid, nx=2, dx=0.05, precision=precision)
    rho = np.full((2, 4, 6), 1.1)
    s.set_material(rho)
    psi = random_state((ng, 2, 2, 2, 4, 6), seed=3)
    s.write_psi(0, psi)
    s.substep_energy(0.025, 1)
    ref, e, _ = orc.Oracle(grid).energy_substep(0.025, rho[1], psi, None)
    assert _relerr(s.read_psi(0), ref) < tol
    s.close()


@pytest.mark.parametrize("cols", [4, 8])
def test_widest_rows(orc, cols):
    """nz = 1024, the widest row the library accepts: nine segments with halo
    lanes per row, against the oracle's transport."""
    grid = _grid(3, 1024, 4, 4, 1)
    s = binding.Solver(grid, nx=1, dx=0.05, precision="fp64")
    s.set_tuning(transport_cols=cols)
    psi = random_state((1, 2, 4, 4, 3, 1024), seed=8)
    s.write_psi(0, psi)
    s.substep_transport(0.3)
    assert _relerr(s.read_psi(0), orc.Oracle(grid).transport_substep(0.3, psi)) < 1e-12
    s.close()
