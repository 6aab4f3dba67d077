"""Lateral domain decomposition of one beam on the GPU (Remark 2): the beam's
rows split into parts, each a context with four halo rows per interior side,
marched in lock-step with halo copies before every transport substep
(pbs_domain_step), or stage by stage with the rows packed and unpacked by
pbs_copy_rows (the multi-process form, here with both parts in one
process).  Every part's own rows of psi equal the undivided march bit for
bit; dose and fluence equal it up to the order of the FP64 tally's atomic
sums; the FP64 result also equals the oracle."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.domain import Domain, assemble_rows, halo_plan, split_rows

pytestmark = pytest.mark.gpu


def _grid(ny, nz, nu, ng):
    return dict(ny=ny, nz=nz, nu=nu, nv=nu, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15,
                e_faces=np.linspace(0.0, 60.0, ng + 1))


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


BEAM = dict(e0=50.0, sigma_e=1.0, sigma_y=0.35, sigma_z=0.3, y0=0.12, z0=-0.05)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _whole(grid, nx, dx, K, precision, rho, steps):
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=K, precision=precision)
    s.set_material(rho)
    s.launch_beam(**BEAM)
    for n in steps:
        s.step(n)
    out = dict(psi=[s.read_psi(k) for k in range(K + 1)], dose=s.read_dose(), fluence=s.read_fluence())
    s.close()
    return out


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
@pytest.mark.parametrize("n_parts,ny", [(2, 22), (3, 25)])
def test_domain_step_equals_undivided_march(orc, precision, n_parts, ny):
    # nz = 8: every part's ny * nz is a multiple of 8, like the whole grid's,
    # so parts and whole run the same kernel forms (the tensor-core source
    # contraction needs it)
    nz, nu, ng, K, nx, dx = 8, 8 if precision != "mixed" else 16, 18, 1, 6, 0.05
    grid = _grid(ny, nz, nu, ng)
    rho = np.random.default_rng(5).uniform(0.5, 1.6, size=(nx, ny, nz))
    ref = _whole(grid, nx, dx, K, precision, rho, (2, nx - 2))
    dom = Domain(grid, nx, dx, n_parts, n_scatter=K, precision=precision)
    dom.set_material(rho)
    dom.launch_beam(**BEAM)
    dom.step(2)
    dom.step(nx - 2)
    for k in range(K + 1):
        assert np.array_equal(dom.read_psi(k), ref["psi"][k]), k
    assert _relerr(dom.read_dose(), ref["dose"]) < 1e-13
    assert _relerr(dom.read_fluence(), ref["fluence"]) < 1e-13
    if precision == "fp64":
        o = orc.Oracle(grid).march(rho, nx, dx, beam=BEAM, n_scatter=K)
        assert _relerr(dom.read_dose(), o["dose"]) < 1e-10
    dom.close()


def test_staged_exchange_equals_domain_step():
    """The multi-process form in one process: each part marched stage by
    stage, halo rows packed into a device buffer by the sending part and
    unpacked by the receiving one (the messages of halo_plan), gives the
    same psi as pbs_domain_step."""
    import torch
    ny, nz, nu, ng, K, nx, dx = 21, 12, 8, 14, 0, 5, 0.05
    grid = _grid(ny, nz, nu, ng)
    rho = np.random.default_rng(8).uniform(0.5, 1.6, size=(nx, ny, nz))
    ref = _whole(grid, nx, dx, K, "fp64", rho, (nx,))
    lay = split_rows(ny, 2)
    parts = []
    for x in lay:
        s = binding.Solver(dict(grid, ny=x.ny), nx=nx, dx=dx, n_scatter=K, precision="fp64")
        s.set_lateral_part(x.y_offset, ny, x.halo_lo, x.halo_hi)
        s.set_material(rho[:, x.y_offset:x.y_offset + x.ny])
        s.launch_beam(**BEAM)
        parts.append(s)

    def exchange():
        for r, s in enumerate(parts):
            for m in halo_plan(lay, r):
                back = [b for b in halo_plan(lay, m.peer) if b.peer == r][0]
                buf = torch.empty(s.n_planes * m.n_recv * nz, dtype=torch.float64, device="cuda")
                parts[m.peer].copy_rows(back.send_first, back.n_send, True, buf)
                s.copy_rows(m.recv_first, m.n_recv, False, buf)

    for _ in range(nx):
        for s in parts:
            s.step_stage(0)
        exchange()
        for s in parts:
            s.step_stage(1)
            s.step_stage(2)
        exchange()
        for s in parts:
            s.step_stage(3)
    psi = assemble_rows(lay, [s.read_psi(0) for s in parts])
    assert np.array_equal(psi, ref["psi"][0])
    assert _relerr(assemble_rows(lay, [s.read_dose() for s in parts]), ref["dose"]) < 1e-13
    for s in parts:
        s.close()


def test_domain_step_rejects_bad_layouts_and_states():
    ny, nz, nu, ng, nx, dx = 20, 8, 4, 8, 3, 0.05
    grid = _grid(ny, nz, nu, ng)
    rho = np.ones((nx, ny, nz))
    dom = Domain(grid, nx, dx, 2, precision="fp64")
    dom.set_material(rho)
    dom.launch_beam(**BEAM)
    a, b = dom.parts
    with pytest.raises(binding.PbsError):  # out of order
        binding.pbs_domain_step([b.ctx, a.ctx], 1)
    with pytest.raises(binding.PbsError):  # one part does not cover the grid
        binding.pbs_domain_step([a.ctx], 1)
    with pytest.raises(binding.PbsError):  # beyond the material
        dom.step(nx + 1)
    # the Crank-Nicolson transport sweeps whole rows: no finite halo
    for s in dom.parts:
        s.set_options(transport_integrator="cn")
    with pytest.raises(binding.PbsError) as e:
        dom.step(1)
    assert e.value.status == -6
    for s in dom.parts:
        s.set_options(transport_integrator="heun")
    # staged steps run in order, and a half-done step blocks the others
    with pytest.raises(binding.PbsError):
        a.step_stage(1)
    a.step_stage(0)
    with pytest.raises(binding.PbsError):
        a.step(1)
    with pytest.raises(binding.PbsError):
        dom.step(1)
    for st in (1, 2, 3):
        a.step_stage(st)
    dom.close()
    # halos thinner than the transport's reach, or on an outer side
    s = binding.Solver(_grid(12, nz, nu, ng), nx=nx, dx=dx, precision="fp64")
    with pytest.raises(binding.PbsError):
        s.set_lateral_part(0, 20, 2, 2)       # halo at the grid's lower edge
    with pytest.raises(binding.PbsError):
        s.set_lateral_part(10, 20, 2, 2)      # rows beyond the grid
    s.set_lateral_part(8, 20, 2, 0)           # accepted alone ...
    s2 = binding.Solver(_grid(12, nz, nu, ng), nx=nx, dx=dx, precision="fp64")
    s2.set_lateral_part(0, 20, 0, 2)
    for x in (s, s2):
        x.set_material(np.ones((nx, x.ny, nz)))
        x.launch_beam(**BEAM)
    with pytest.raises(binding.PbsError):     # ... but 2 halo rows are too few to step
        binding.pbs_domain_step([s2.ctx, s.ctx], 1)
    s.close()
    s2.close()
