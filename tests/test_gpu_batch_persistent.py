"""The persistent batch (pbs_run_batch): several beams, each its own context
with its own lateral grid, energy groups and depth, marched by one launch
with a device queue of tiles and per-beam completion counters.

* Every beam's psi equals its own march (pbs_run with the same kernel forms)
  bit for bit; dose and fluence up to the order of the atomic FP64 sums.
* Reduced spots of the batched-spot recipe against the FP64 oracle (FP32
  march tolerance, 1e-4 of the maximum dose).
* A graph-recorded batch replays to the same result.
* Failure detection without a GPU fault: a hold that nothing releases
  (hold_beam) makes the bounded device waits run out after 50 ms; the next
  synchronising call returns PBS_ERR_TIMEOUT, and a new batch on the same
  contexts runs correctly."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding

pytestmark = pytest.mark.gpu

FORMS = dict(energy_angles=8, energy_form=1, angular_form=2, transport_cols=4)


def _relerr(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


# (lateral ny, nz, groups, top energy, beam energy, depth steps, lateral offset)
BEAMS = [(8, 8, 24, 40.0, 35.0, 9, 0.0), (12, 16, 31, 52.0, 47.0, 14, 0.07), (10, 12, 18, 30.0, 26.0, 5, -0.05),
         (16, 8, 40, 64.0, 60.0, 12, 0.0)]


def _make(spec, precision, nu=8, seed=0):
    ny, nz, ng, emax, e0, steps, y0 = spec
    grid = dict(ny=ny, nz=nz, nu=nu, nv=nu, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
                e_faces=np.linspace(0.0, emax, ng + 1))
    s = binding.Solver(grid, nx=steps, dx=0.05, precision=precision)
    s.set_tuning(**FORMS)
    rho = np.random.default_rng(seed).uniform(0.6, 1.5, size=(steps, ny, nz))
    s.set_material(rho)
    beam = dict(e0=e0, sigma_e=1.0, sigma_y=0.3, sigma_z=0.25, y0=y0)
    s.launch_beam(**beam)
    return s, grid, rho, beam


def _results(s):
    return s.read_psi(0), s.read_dose(), s.read_fluence()


@pytest.mark.parametrize("precision,use_graph,shape,cols,pipeline", [
    ("fp32", False, 0, 0, 0), ("fp32", True, 0, 0, 1), ("mixed", False, 0, 0, 0), ("mixed", True, 1, 6, 1),
    ("fp32", False, 1, 4, 0), ("fp32", False, 1, 6, 1)])
def test_batch_equals_each_beams_own_march(precision, use_graph, shape, cols, pipeline):
    """Both CTA shapes, both transport column counts, whole and pipelined
    passes: every variant runs the same arithmetic per cell."""
    ref = []
    for i, spec in enumerate(BEAMS):
        s, *_ = _make(spec, precision, seed=i)
        s.run(use_graph=False)
        ref.append(_results(s))
        s.close()
    solvers = [_make(spec, precision, seed=i)[0] for i, spec in enumerate(BEAMS)]
    ws = binding.run_batch(solvers, use_graph=use_graph, shape=shape, transport_cols=cols, pipeline=pipeline)
    for s, (psi, dose, flu) in zip(solvers, ref):
        assert s.depth == s.nx
        got = _results(s)
        assert np.array_equal(got[0], psi)
        assert _relerr(got[1], dose) < 1e-13
        assert _relerr(got[2], flu) < 1e-13
    if use_graph:  # a replay of the recorded batch restarts every beam and gives the same
        binding.run_batch(solvers, use_graph=True, workspace=ws, shape=shape, transport_cols=cols, pipeline=pipeline)
        for s, (psi, dose, _) in zip(solvers, ref):
            assert np.array_equal(s.read_psi(0), psi)
            assert _relerr(s.read_dose(), dose) < 1e-13
    for s in solvers:
        s.close()


@pytest.mark.parametrize("pipeline", [0, 1])
def test_single_beam_with_16x16_angles(pipeline):
    """One beam with 16 x 16 angles (shape 0, one angular block per CTA),
    enough groups for several 32-stack chunks of a pipelined pass."""
    spec = (8, 12, 40, 64.0, 60.0, 7, 0.04)
    s, *_ = _make(spec, "fp32", nu=16)
    s.run(use_graph=False)
    ref = _results(s)
    s.close()
    t, *_ = _make(spec, "fp32", nu=16)
    binding.run_batch([t], shape=0, pipeline=pipeline)
    got = _results(t)
    assert np.array_equal(got[0], ref[0])
    assert _relerr(got[1], ref[1]) < 1e-13
    with pytest.raises(binding.PbsError) as e:
        binding.run_batch([t], shape=1)
    assert e.value.status == -6
    t.close()


def test_batch_autotuner_picks_a_shape_and_restarts_the_beams():
    ref = []
    for i, spec in enumerate(BEAMS):
        s, *_ = _make(spec, "fp32", seed=i)
        s.run(use_graph=False)
        ref.append(s.read_psi(0))
        s.close()
    solvers = [_make(spec, "fp32", seed=i)[0] for i, spec in enumerate(BEAMS)]
    opts, ws = binding.autotune_batch(solvers, steps=3)
    assert opts["shape"] in (0, 1) and opts["transport_cols"] in (4, 6) and opts["pipeline"] in (0, 1)
    assert all(s.depth == 0 for s in solvers)  # restarted from the projections
    binding.run_batch(solvers, workspace=ws, **opts)
    for s, psi in zip(solvers, ref):
        assert np.array_equal(s.read_psi(0), psi)
        s.close()


def test_batch_of_reduced_spots_matches_oracle():
    """Spots of the batched recipe (energy-dependent groups and depth, 8x8
    angles in +-0.1) on a reduced 12x12 lateral grid, each against the FP64
    oracle's march of the same beam."""
    import oracle
    from paper_2504_00340_gb300.workloads import spot_batch
    spots = [w for w in spot_batch(n_beams=256) if w.beam["e0"] < 95.0][:3]
    solvers, refs = [], []
    for w in spots:
        ng = max(8, w.ng // 4)
        grid = dict(ny=12, nz=12, nu=8, nv=8, dy=0.1, dz=0.1, u_max=0.1, v_max=0.1,
                    e_faces=np.linspace(0.0, w.e_max, ng + 1))
        steps = 30
        beam = {k: v for k, v in w.beam.items() if k not in ("yc", "zc")}
        s = binding.Solver(grid, nx=steps, dx=w.dx, precision="mixed")
        s.set_material(np.ones((steps, 12, 12)))
        s.launch_beam(**beam)
        solvers.append(s)
        refs.append(oracle.Oracle(grid).march(np.ones((steps, 12, 12)), steps, w.dx, beam=beam))
    binding.run_batch(solvers)
    for s, r in zip(solvers, refs):
        assert _relerr(s.read_dose(), r["dose"]) < 1e-4
        assert _relerr(s.read_fluence(), r["fluence"]) < 1e-4
        s.close()


def test_batch_wait_that_runs_out_reports_timeout_and_recovers():
    ref = []
    for i, spec in enumerate(BEAMS[:3]):
        s, *_ = _make(spec, "fp32", seed=i)
        s.run(use_graph=False)
        ref.append(s.read_dose())
        s.close()
    solvers = [_make(spec, "fp32", seed=i)[0] for i, spec in enumerate(BEAMS[:3])]
    ws = binding.run_batch(solvers, wait_limit_ms=50.0, hold_beam=1)
    for s in solvers:
        with pytest.raises(binding.PbsError) as e:
            s.read_dose()
        assert e.value.status == -5
    binding.run_batch(solvers, workspace=ws)
    for s, d in zip(solvers, ref):
        assert _relerr(s.read_dose(), d) < 1e-13
        s.close()


def test_batch_rejects_what_it_does_not_handle():
    s_ok, *_ = _make(BEAMS[0], "fp32")
    s64, *_ = _make(BEAMS[1], "fp64")
    with pytest.raises(binding.PbsError) as e:
        binding.run_batch([s_ok, s64])
    assert e.value.status == -6
    s16, *_ = _make(BEAMS[2], "fp32", nu=16)
    with pytest.raises(binding.PbsError):
        binding.run_batch([s_ok, s16])   # another angle grid
    with pytest.raises(binding.PbsError):
        binding.run_batch([s_ok, s_ok])  # the same context twice
    for s in (s_ok, s64, s16):
        s.close()
