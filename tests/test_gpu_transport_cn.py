"""GPU parity of the second transport integrator (Remark 3: Crank-Nicolson
with the slope taken from the old state in the implicit half, solved by an
upwind sweep) against the oracle: single substeps over plane shapes that
exercise the lane layout (columns per lane 4, 6, 8, ragged last lane, one-row
and one-column planes), a Courant number far beyond the explicit limit, and a
whole march."""
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


SHAPES = [(9, 16, 4, 4), (12, 37, 4, 4), (7, 96, 6, 4), (5, 130, 4, 6), (6, 200, 2, 2), (4, 256, 2, 2),
          (1, 24, 4, 4), (10, 1, 4, 4), (2, 3, 2, 2)]


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 5e-6)])
@pytest.mark.parametrize("ny,nz,nu,nv", SHAPES)
def test_cn_transport_substep(orc, precision, tol, ny, nz, nu, nv):
    grid = _grid(ny, nz, nu, nv, 2)
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision)
    s.set_options(transport_integrator="cn")
    psi = random_state((2, 2, nv, nu, ny, nz), seed=ny * 131 + nz)
    s.write_psi(0, psi)
    s.substep_transport(0.3)
    o = orc.Oracle(grid)
    o.set_transport_cn(True)
    ref = o.transport_substep(0.3, psi)
    assert _relerr(s.read_psi(0), ref) < tol
    heun = orc.Oracle(grid).transport_substep(0.3, psi)
    assert _relerr(heun, ref) > 1e3 * tol  # the two integrators really differ
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-5)])
def test_cn_transport_large_courant(orc, precision, tol):
    """h |u| / dy = 3 in both directions: ten substeps stay bounded and
    equal the oracle's."""
    grid = _grid(20, 24, 2, 2, 1, u_max=0.3)
    s = binding.Solver(grid, nx=1, dx=0.05, precision=precision)
    s.set_options(transport_integrator="cn")
    o = orc.Oracle(grid)
    o.set_transport_cn(True)
    h = 3.0 * 0.1 / 0.1  # |u| = 0.1 for 2 nodes in +-0.3
    psi = np.abs(random_state((1, 2, 2, 2, 20, 24), seed=7))
    s.write_psi(0, psi)
    ref = psi
    for _ in range(10):
        s.substep_transport(h)
        ref = o.transport_substep(h, ref)
    got = s.read_psi(0)
    assert _relerr(got, ref) < tol
    assert np.abs(got).max() < 1.5 * np.abs(psi).max()
    s.close()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_march_with_cn_transport(orc, precision, tol):
    grid = _grid(14, 18, 8, 8, 24)
    nx, dx = 7, 0.05
    rho = np.random.default_rng(12).uniform(0.5, 1.5, size=(nx, 14, 18))
    beam = dict(e0=45.0, sigma_e=1.0, sigma_y=0.25, sigma_z=0.2, y0=0.05)
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision)
    s.set_options(transport_integrator="cn")
    s.set_material(rho)
    s.launch_beam(**beam)
    s.step(nx)
    o = orc.Oracle(grid)
    o.set_transport_cn(True)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
    assert _relerr(s.read_dose(), ref["dose"]) < tol
    assert _relerr(s.read_fluence(), ref["fluence"]) < tol
    s.close()


def test_cn_transport_row_limit():
    s = binding.Solver(_grid(4, 300, 2, 2, 2), nx=1, dx=0.05, precision="fp32")
    with pytest.raises(binding.PbsError):
        s.set_options(transport_integrator="cn")
    s.set_options(transport_integrator="heun")
    s.close()
