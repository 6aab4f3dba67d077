"""The allocation-free source evaluation (pbs_eval_source_noalloc) against the
context path (pbs_eval_source) on the same FP32 state, two calls in a row.

Callers of this entry point cannot allocate device memory; the test itself
allocates its input and output buffers with torch (as such a caller's host
framework would) and passes raw device pointers, while the entry point keeps
its scratch in the library's own file-scope device array."""
import numpy as np
import pytest

from paper_2504_00340_gb300 import binding
from paper_2504_00340_gb300.workloads import smooth_state

pytestmark = pytest.mark.gpu


def test_noalloc_source_matches_context_path():
    import torch
    torch.cuda.set_device(0)
    ny, nz, nu, nv, ng = 9, 8, 8, 8, 20
    grid = dict(ny=ny, nz=nz, nu=nu, nv=nv, dy=0.1, dz=0.1, u_max=0.15, v_max=0.15,
                e_faces=np.linspace(0.0, 60.0, ng + 1))
    phys = dict(binding.DEFAULT_PHYSICS)
    rho = np.random.default_rng(1).uniform(0.3, 1.9, size=(2, ny, nz))
    s = binding.Solver(grid, nx=2, dx=0.05, n_scatter=1, precision="fp32", physics=phys)
    s.set_material(rho)
    p2 = torch.as_tensor(s.tables()["p2"], dtype=torch.float32, device="cuda").contiguous()
    stream = torch.cuda.current_stream()
    for call, seed in enumerate((3, 4)):
        psi = smooth_state(ny, nz, ng, nv, nu, seed=seed)
        s.write_psi(0, psi)
        ref = s.eval_source(0, 1)
        psi_dev = s.psi_view(0).contiguous()
        rho_dev = torch.as_tensor(rho[1], dtype=torch.float32, device="cuda").contiguous()
        out = torch.full((ng, nv, nu, ny, nz), float("nan"), dtype=torch.float32, device="cuda")
        binding.pbs_eval_source_noalloc(psi_dev.data_ptr(), rho_dev.data_ptr(), p2.data_ptr(), grid["e_faces"],
                                        ng, nu, nv, ny, nz, grid["u_max"], grid["v_max"], phys["sigma_ct"],
                                        phys["lambda_p1"], out.data_ptr(), stream.cuda_stream)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        assert np.isfinite(got).all(), call
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err < 1e-6, (call, err)
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
