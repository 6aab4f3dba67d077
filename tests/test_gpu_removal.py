"""GPU parity with a group-dependent catastrophic removal sigma_c,t,g
(Section 4; Remark 1): the library's tables come in through pbs_set_tables
with a removal cross section that varies by two orders of magnitude across
the groups, the oracle gets the same table, and the two must agree.  With a
constant sigma a kernel that used the receiving group's sigma in the source,
or a neighbouring group's sigma in the removal term, would pass every other
test; here it cannot.  Tolerances as in test_gpu_parity: FP64 substeps 1e-12
and marches 1e-10 relative to the maximum, FP32 substeps 2e-6, FP32 march
1e-4, mixed (BF16 source contraction) 1e-3 of the maximum dose."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.workloads import smooth_state

pytestmark = pytest.mark.gpu


def _grid(ny, nz, nu, nv, ng, e_max=60.0):
    return dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15,
                e_faces=np.linspace(0.0, e_max, ng + 1))


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _sigma_table(ng, seed):
    return 10.0 ** np.random.default_rng(seed).uniform(-3.0, -1.0, size=ng)


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def _pair(orc, grid, nx, dx, K, precision, sig, rho):
    """A library context and an oracle with the same group-dependent sigma:
    the oracle's own tables with sig replacing the removal column, handed to
    the library through pbs_set_tables."""
    lam = 0.05
    o = orc.Oracle(grid, dict(lambda_p1=lam))
    o.set_sigma(sig)
    t = o.tables()
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=K, precision=precision)
    s.set_tables(t["s_face"], t["ts"], sig, lam, t["p2"])
    got = s.tables()
    assert _relerr(got["sig"], sig) == 0.0
    assert _relerr(got["p1"], t["p1"]) < 1e-13
    s.set_material(rho)
    return s, o


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 2e-6)])
@pytest.mark.parametrize("ny,nz", [(6, 7), (5, 8)])
def test_energy_substep_source_chain_with_group_dependent_sigma(orc, precision, tol, ny, nz):
    """E(h) on three components chained by their sources (odd and even
    lateral counts: the one-lane and the packed FP32 kernels), 33 groups."""
    ng, K = 33, 2
    grid = _grid(ny, nz, 4, 4, ng)
    rho = np.random.default_rng(3).uniform(0.3, 1.9, size=(3, ny, nz))
    sig = _sigma_table(ng, seed=21)
    s, o = _pair(orc, grid, 3, 0.05, K, precision, sig, rho)
    states = [smooth_state(ny, nz, ng, 4, 4, seed=30 + k) for k in range(K + 1)]
    for k in range(K + 1):
        s.write_psi(k, states[k])
    h, slab = 0.4, 2
    s.substep_energy(h, slab, fluence_plane=-1)
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
    assert _relerr(dose, edep / (rho[slab] * 0.05 * 0.1 * 0.1)) < 10 * tol
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_source_with_group_dependent_sigma(orc, precision):
    """The catastrophic source alone (the fused R recursion and the angle
    contraction) with the emitting group's sigma."""
    ny, nz, ng = 9, 8, 20
    grid = _grid(ny, nz, 16, 16, ng) if precision == "mixed" else _grid(ny, nz, 8, 8, ng)
    na_u = grid["nu"]
    rho = np.random.default_rng(4).uniform(0.3, 1.9, size=(1, ny, nz))
    sig = _sigma_table(ng, seed=22)
    s, o = _pair(orc, grid, 1, 0.05, 1, precision, sig, rho)
    psi = smooth_state(ny, nz, ng, na_u, na_u, seed=5)
    s.write_psi(0, psi)
    got = s.eval_source(0, 0)
    ref = o.source(rho[0], psi)
    tol = {"fp64": 1e-12, "fp32": 1e-6, "mixed": 8e-3}[precision]
    assert _relerr(got, ref) < tol
    s.close()


@pytest.mark.parametrize("precision,tol,nu", [("fp64", 1e-10, 8), ("fp32", 1e-4, 8), ("mixed", 1e-3, 16)])
def test_march_k2_with_group_dependent_sigma(orc, precision, tol, nu):
    """A K = 2 march (primary and two scattered components) through a
    heterogeneous density with the varying sigma: dose, fluence and every
    component against the oracle's march."""
    ny = nz = 10
    ng, nx, dx = 30, 12, 0.05
    grid = _grid(ny, nz, nu, nu, ng)
    rho = np.random.default_rng(6).uniform(0.5, 1.6, size=(nx, ny, nz))
    sig = _sigma_table(ng, seed=23) * 3.0  # up to 0.3 cm^2/g: the scattered fields carry visible weight
    s, o = _pair(orc, grid, nx, dx, 2, precision, sig, rho)
    beam = dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)
    s.launch_beam(**beam)
    s.step(nx)
    ref = o.march(rho, nx, dx, beam=beam, n_scatter=2)
    assert _relerr(s.read_dose(), ref["dose"]) < tol
    assert _relerr(s.read_fluence(), ref["fluence"]) < tol
    for k in range(3):
        ktol = tol if precision != "mixed" else 1e-2
        assert _relerr(s.read_psi(k), ref["psi"][k]) < ktol, k
    # the scattered components carry protons (each is compared against its own
    # maximum above): particle counts sum(psi^1 dE) relative to the primary's
    de = np.diff(grid["e_faces"])[:, None, None, None, None]
    count = [float((ref["psi"][k][:, 0] * de).sum()) for k in range(3)]
    assert count[1] > 1e-4 * count[0] and count[2] > 1e-8 * count[0], count
    s.close()
