"""GPU parity of batched contexts (several beams on one grid marching in
lock-step), per-beam depth ranges, the whole-march CUDA graph and the launch
autotuner.  Every beam of a batch must reproduce the oracle's march of that
beam alone, and the graph and any tuned launch shape must reproduce the
plain launch sequence."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding

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


BEAMS = [dict(e0=50.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.25, y0=0.05),
         dict(e0=42.0, sigma_e=0.8, sigma_y=0.2, sigma_z=0.3, z0=-0.2),
         dict(e0=35.0, sigma_e=1.2, sigma_y=0.35, sigma_z=0.2, y0=-0.1, z0=0.1)]


def test_batch_matches_oracle_per_beam_fp64(orc):
    """Three different beams (K = 1) in one context: each beam's dose, fluence
    and psi equal the oracle's single-beam march within 1e-10."""
    grid = _grid(14, 10, 8, 8, 24)
    nx, dx = 8, 0.05
    rho = np.random.default_rng(3).uniform(0.4, 1.8, size=(nx, 14, 10))
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64", n_beams=3)
    s.set_material(rho)
    s.launch_beams(BEAMS)
    s.step(3)
    s.step(nx - 3)
    dose, flu = s.read_dose(), s.read_fluence()
    assert dose.shape == (3, nx, 14, 10) and flu.shape == (3, nx + 1, 14, 10)
    o = orc.Oracle(grid)
    for b, beam in enumerate(BEAMS):
        ref = o.march(rho, nx, dx, beam=beam, n_scatter=1)
        assert _relerr(dose[b], ref["dose"]) < 1e-10, b
        assert _relerr(flu[b], ref["fluence"]) < 1e-10, b
        for j in range(2):
            assert _relerr(s.read_psi(2 * b + j), ref["psi"][j]) < 1e-10, (b, j)
    s.close()


def test_per_beam_depths(orc):
    """Beams with their own depth ranges (non-increasing): beam b marches
    steps[b] steps and then only gets its closing half; its dose equals the
    oracle's march of steps[b] steps, zero beyond."""
    grid = _grid(10, 12, 8, 8, 20)
    nx, dx = 7, 0.05
    steps = [7, 5, 5, 2]
    beams = BEAMS + [dict(e0=30.0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.3)]
    rho = np.random.default_rng(4).uniform(0.5, 1.5, size=(nx, 10, 12))
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp64", n_beams=4)
    s.set_material(rho)
    s.set_beam_steps(steps)
    s.launch_beams(beams)
    s.step(2)
    s.step(nx - 2)
    dose, flu = s.read_dose(), s.read_fluence()
    o = orc.Oracle(grid)
    for b, beam in enumerate(beams):
        n = steps[b]
        ref = o.march(rho[:n], n, dx, beam=beam, n_scatter=1)
        assert _relerr(dose[b, :n], ref["dose"]) < 1e-10, b
        assert not dose[b, n:].any(), b
        assert _relerr(flu[b, :n + 1], ref["fluence"]) < 1e-10, b
        assert not flu[b, n + 1:].any(), b
        assert _relerr(s.read_psi(2 * b), ref["psi"][0]) < 1e-10, b
    s.close()


def test_beam_steps_validation():
    grid = _grid(4, 4, 4, 4, 8)
    s = binding.Solver(grid, nx=5, dx=0.05, precision="fp32", n_beams=3)
    for bad in ([5, 6, 1], [1, 2, 3], [5, 5, -1], [5, 5]):
        with pytest.raises(binding.PbsError):
            s.set_beam_steps(bad)
    s.set_beam_steps([5, 3, 3])
    s.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32", "mixed"])
def test_graph_run_equals_launch_sequence(precision):
    """pbs_run with a recorded graph (replayed twice) and without one give the
    same dose, fluence and psi as launch_beams + step + flush."""
    grid = _grid(12, 16, 16, 16, 16) if precision == "mixed" else _grid(12, 16, 8, 8, 16)
    nx, dx = 6, 0.05
    rho = np.random.default_rng(5).uniform(0.5, 1.5, size=(nx, 12, 16))
    steps = [6, 4, 1]

    def make():
        s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision=precision, n_beams=3)
        s.set_material(rho)
        s.set_beam_steps(steps)
        s.launch_beams(BEAMS)
        return s

    a = make()
    a.step(nx)
    ref = (a.read_dose(), a.read_fluence(), a.read_psi(0), a.read_psi(3))
    a.close()
    tol = 1e-12 if precision == "fp64" else 1e-6
    for use_graph in (False, True):
        s = make()
        for _ in range(2):
            s.run(use_graph)
            got = (s.read_dose(), s.read_fluence(), s.read_psi(0), s.read_psi(3))
            for x, y in zip(got, ref):
                assert _relerr(x, y) < tol
        assert s.depth == nx
        s.close()


def test_graph_rerecords_after_depth_change():
    grid = _grid(8, 8, 8, 8, 12)
    nx, dx = 5, 0.05
    s = binding.Solver(grid, nx=nx, dx=dx, precision="fp32", n_beams=2)
    s.set_material(np.ones((nx, 8, 8)))
    s.launch_beams(BEAMS[:2])
    s.run(True)
    d5 = s.read_dose()
    s.launch_beams(BEAMS[:2])
    s.set_beam_steps([3, 3])
    s.run(True)
    d3 = s.read_dose()
    assert s.depth == 3
    assert not d3[:, 3:].any()
    assert _relerr(d3[:, :3], d5[:, :3]) < 1e-5
    s.close()


def test_autotune_and_forms_keep_results():
    """The tuner picks shapes and forms from its candidate sets and restarts
    the beams.  Shapes within one kernel form give the same psi bit for bit;
    the packed and TMA forms agree with the plain ones to FP32 rounding."""
    grid = _grid(16, 32, 8, 8, 20)
    nx, dx = 4, 0.05
    rho = np.random.default_rng(6).uniform(0.5, 1.5, size=(nx, 16, 32))
    s = binding.Solver(grid, nx=nx, dx=dx, precision="fp32", n_beams=2)
    s.set_material(rho)
    s.launch_beams(BEAMS[:2])
    s.autotune(2)
    t = s.tuning
    assert t["energy_angles"] in (4, 8, 16) and t["energy_form"] in (0, 1)
    assert t["transport_ctas"] in (0, 1, 2, 3, 4) and t["angular_form"] in (0, 1, 2, 3, 4, 5, 6, 7)
    assert t["transport_cols"] in (4, 6, 8)
    assert s.depth == 0
    plain = dict(energy_angles=8, energy_form=0, transport_ctas=0, angular_form=0)
    shapes = [plain, dict(energy_angles=4, energy_form=0, transport_ctas=1, angular_form=0),
              dict(energy_angles=16, energy_form=1, transport_ctas=3, angular_form=2),
              dict(energy_angles=8, energy_form=1, transport_ctas=0, angular_form=1), t]
    out = []
    for shape in shapes:
        s.set_tuning(**shape)
        s.launch_beams(BEAMS[:2])
        s.step(nx)
        out.append((s.read_dose(), s.read_psi(0), s.read_psi(1)))
    base = out[0]
    for shape, got in zip(shapes, out):
        same_forms = shape["energy_form"] == 0 and shape["angular_form"] == 0
        for j in (1, 2):
            if same_forms:
                assert np.array_equal(got[j], base[j]), shape
            else:
                assert _relerr(got[j], base[j]) < 2e-5, shape
        assert _relerr(got[0], base[0]) < 2e-5, shape
    with pytest.raises(binding.PbsError):
        s.set_tuning(energy_angles=6)
    with pytest.raises(binding.PbsError):
        s.set_tuning(energy_angles=8, angular_form=8)
    s.close()


def test_large_batch_chunked_launches():
    """130 beams x 512 groups (K = 1): the angular and CUDA-core source grids
    exceed 65535 blocks in one dimension and go in chunks; beams 0, 64, 129
    equal single-beam contexts of the same beam."""
    grid = _grid(8, 8, 8, 8, 512, e_max=120.0)
    nx, dx, B = 2, 0.05, 130
    rho = np.full((nx, 8, 8), 1.0)
    beams = [dict(e0=60.0 + 0.3 * b, sigma_e=1.0, sigma_y=0.25, sigma_z=0.25, y0=0.01 * (b % 7)) for b in range(B)]
    s = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp32", n_beams=B)
    s.set_material(rho)
    s.launch_beams(beams)
    s.step(nx)
    dose = s.read_dose()
    for b in (0, 64, 129):
        one = binding.Solver(grid, nx=nx, dx=dx, n_scatter=1, precision="fp32")
        one.set_material(rho)
        one.launch_beam(**beams[b])
        one.step(nx)
        assert _relerr(dose[b], one.read_dose()) < 1e-5, b
        for j in range(2):
            assert np.array_equal(s.read_psi(2 * b + j), one.read_psi(j)), (b, j)
        one.close()
    s.close()


def test_spot_bucket_path_matches_oracle(orc):
    """Reduced spots of the seeded batch (same recipe, lower energies and a
    16 x 16 lateral grid so that the oracle finishes in seconds) through the
    planner, the autotuner and the recorded-graph bucket march, mixed
    precision: each spot's dose against the oracle's march of that spot on the
    bucket's energy grid, within 1e-3 of its maximum."""
    from paper_2504_00340_gb300 import spots as S
    from paper_2504_00340_gb300.workloads import spot_batch
    base = spot_batch(n_beams=4)
    red = []
    for i, e0 in enumerate((40.0, 38.0, 35.0, 31.0)):
        rng_cm = 0.0022 * e0 ** 1.77
        n = int(np.ceil((rng_cm + 0.3) / 0.05))
        beam = dict(base[i].beam, e0=e0, sigma_y=0.2, sigma_z=0.2)
        red.append(base[i].with_(name=f"red{i}", ny=16, nz=16, ng=int(np.ceil(e0 / 1.0)), e_max=e0 + 4.0,
                                 n_steps=n, beam=beam))
    buckets = S.plan_buckets(red, max_waste=0.3)
    assert sum(len(b.members) for b in buckets) == 4 and len(buckets) <= 2
    for b in buckets:
        doses, ms, kernels, tuning = S.run_bucket(b, red, use_graph=True, autotune=True)
        assert ms > 0 and kernels > 0
        grid = S.bucket_grid(b, red)
        o = orc.Oracle(grid)
        for j, i in enumerate(b.members):
            w = red[i]
            beam = {k: v for k, v in w.beam.items() if k not in ("yc", "zc")}
            ref = o.march(np.ones((w.n_steps, 16, 16)), w.n_steps, w.dx, beam=beam, n_scatter=0)
            d = doses[i]
            assert d.shape == ref["dose"].shape
            assert np.abs(d - ref["dose"]).max() / np.abs(ref["dose"]).max() < 1e-3, i
