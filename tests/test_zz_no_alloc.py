"""The allocation-free source evaluation (pbs_eval_source_noalloc) against the
context path (pbs_eval_source) and the FP64 oracle on the same FP32 state,
two calls in a row.

Callers of this entry point cannot allocate device memory themselves (their
host framework owns the device memory and hands them pre-carved buffers);
the test plays that framework: it allocates the input and output buffers
with torch up front and passes raw device pointers, while the entry point
keeps its scratch in the library's own file-scope device array.  Between the
first call (which loads the library's kernels) and the end of the second,
the device's free memory must not change."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.workloads import smooth_state

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def orc():
    import oracle
    oracle.build()
    return oracle


def test_noalloc_source_matches_context_path_and_oracle(orc):
    import torch
    torch.cuda.set_device(0)
    ny, nz, nu, nv, ng = 9, 8, 8, 8, 20
    grid = dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15,
                e_faces=np.linspace(0.0, 60.0, ng + 1))
    phys = dict(binding.DEFAULT_PHYSICS)
    rho = np.random.default_rng(1).uniform(0.3, 1.9, size=(2, ny, nz))
    s = binding.Solver(grid, nx=2, dx=0.05, n_scatter=1, precision="fp32", physics=phys)
    s.set_material(rho)
    o = orc.Oracle(grid, phys)
    p2 = torch.as_tensor(s.tables()["p2"], dtype=torch.float32, device="cuda").contiguous()
    rho_dev = torch.as_tensor(rho[1], dtype=torch.float32, device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    # every buffer and every reference first: the calls below must run with
    # nothing else allocating on the device
    calls = []
    for seed in (3, 4):
        psi = smooth_state(ny, nz, ng, nv, nu, seed=seed)
        s.write_psi(0, psi)
        psi32 = s.read_psi(0)  # the FP32 state both paths see
        calls.append(dict(
            psi_dev=s.psi_view(0).contiguous().clone(),
            out=torch.full((ng, nv, nu, ny, nz), float("nan"), dtype=torch.float32, device="cuda"),
            ref_ctx=s.eval_source(0, 1),
            ref_orc=o.source(rho[1], psi32)))
    torch.cuda.synchronize()
    free = []
    for c in calls:
        binding.pbs_eval_source_noalloc(c["psi_dev"].data_ptr(), rho_dev.data_ptr(), p2.data_ptr(), grid["e_faces"],
                                        ng, nu, nv, ny, nz, grid["u_max"], grid["v_max"], phys["sigma_ct"],
                                        phys["lambda_p1"], c["out"].data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
    assert free[1] == free[0], "the second call changed the device's free memory"
    for i, c in enumerate(calls):
        got = c["out"].double().cpu().numpy()
        assert np.isfinite(got).all(), i
        err_ctx = np.abs(got - c["ref_ctx"]).max() / np.abs(c["ref_ctx"]).max()
        assert err_ctx < 1e-6, (i, err_ctx)
        # FP32 arithmetic against the FP64 oracle: the same bound as the
        # context path's FP32 source contraction
        err_orc = np.abs(got - c["ref_orc"]).max() / np.abs(c["ref_orc"]).max()
        assert err_orc < 1e-6, (i, err_orc)
    s.close()


def test_noalloc_rejects_oversized_calls():
    import torch
    torch.cuda.set_device(0)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    ef = np.linspace(0.0, 100.0, 65)
    with pytest.raises(binding.PbsError) as e:
        # 64 * 256 * 128 * 128 elements: above the 4 Mi scratch limit
        binding.pbs_eval_source_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), ef, 64, 16, 16, 128,
                                        128, 0.15, 0.15, 0.012, 0.05, dummy.data_ptr(), 0)
    assert e.value.status == -6
    ef = np.linspace(0.0, 100.0, 2050)
    with pytest.raises(binding.PbsError) as e:
        # 2049 groups of one lane each: within the element limit, above the group limit
        binding.pbs_eval_source_noalloc(dummy.data_ptr(), dummy.data_ptr(), dummy.data_ptr(), ef, 2049, 1, 1, 1,
                                        1, 0.15, 0.15, 0.012, 0.05, dummy.data_ptr(), 0)
    assert e.value.status == -6
