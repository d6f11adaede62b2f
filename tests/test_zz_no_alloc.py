"""The entry point that allocates nothing, lbm_residual_sums_noalloc.

Some callers cannot let the library call cudaMalloc while they run (their
device memory comes from their own pool, or their loop must not allocate, or
they record into a CUDA graph).  For them the convergence sums are computed on
their own device buffers with a fixed scratch array inside the library.  This
test checks, through the C ABI, that two calls in a row give the same sums as
the context API's lbm_residual on the same states, and that an oversize domain
is rejected.  It lives in its own file, collected last.
"""
import numpy as np
import pytest

import workloads as wl
from paper_1806_10251_gb300 import lbm

pytestmark = pytest.mark.gpu

W = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)


def _device_populations(torch, solver):
    """The solver's current populations as an FP32 deviation array on the GPU
    (layout [9][ny][nx], pitch nx), built from the host copy."""
    f = solver.populations()
    g = (f - W[:, None, None]).astype(np.float32)
    return torch.from_numpy(np.ascontiguousarray(g)).cuda()


def test_noalloc_sums_match_lbm_residual_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = wl.random_cavity_state(200, 90, 0.5, Re=60.0, seed=12)
    ref = lbm.solver_from_case(case)
    # the context's snapshot after initialisation is the initial velocity field
    _, u0, v0 = ref.fields()
    snap_u = torch.from_numpy(u0).cuda()
    snap_v = torch.from_numpy(v0).cuda()
    sums = torch.zeros(5, dtype=torch.float64, device="cuda")
    desc = lbm.PopulationDesc(case.nx, case.ny, case.nx, lbm.STORAGE_F32, case.gamma, 0.0, 0.0, None)
    for steps in (40, 25):
        ref.step(steps)
        _, expected = ref.residual()
        f_dev = _device_populations(torch, ref)
        lbm.residual_sums_noalloc(desc, f_dev.data_ptr(), snap_u.data_ptr(), snap_v.data_ptr(), sums.data_ptr())
        torch.cuda.synchronize()
        got = sums.cpu().numpy()
        assert np.allclose(got, expected, rtol=1e-12, atol=1e-12), (got, expected)
        # the snapshot now holds the current velocity, as the context's does
        _, u, v = ref.fields()
        assert np.allclose(snap_u.cpu().numpy(), u, rtol=0, atol=1e-15)
        assert np.allclose(snap_v.cpu().numpy(), v, rtol=0, atol=1e-15)


def test_noalloc_pitched_fp16_with_solid_and_force():
    """The descriptor's other paths: a plane pitch above nx (200 cells in rows of
    256), a solid mask on the device, a uniform body force (rho u = sum f e -
    F/(2 gamma)) and FP16 storage (2^14 (f - w) as half).  The populations are
    the context's own, re-encoded from its host copy; the sums must equal
    lbm_residual's on that context on two calls in a row."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = wl.random_cavity_state(200, 90, 0.5, Re=60.0, seed=13)
    case.Fx, case.Fy = 2e-6, -1e-6
    solid = np.zeros((case.ny, case.nx), np.uint8)
    solid[30:52, 80:111] = 1
    case.solid = solid
    ref = lbm.solver_from_case(case, storage=lbm.STORAGE_F16)
    pitch = 256
    _, u0, v0 = ref.fields()
    snap_u = torch.from_numpy(np.nan_to_num(u0)).cuda()
    snap_v = torch.from_numpy(np.nan_to_num(v0)).cuda()
    mask = np.zeros((case.ny, pitch), np.uint8)
    mask[:, :case.nx] = solid
    mask_dev = torch.from_numpy(mask).cuda()
    sums = torch.zeros(5, dtype=torch.float64, device="cuda")
    desc = lbm.PopulationDesc(case.nx, case.ny, pitch, lbm.STORAGE_F16, case.gamma, case.Fx, case.Fy,
                              mask_dev.data_ptr())
    for steps in (30, 17):
        ref.step(steps)
        _, expected = ref.residual()
        f = ref.populations()
        g = np.zeros((9, case.ny, pitch), np.float16)
        g[:, :, :case.nx] = (16384.0 * (f - W[:, None, None])).astype(np.float16)
        # the re-encoding reproduces the host copy to rounding (the stored half values)
        back = g[:, :, :case.nx].astype(np.float64) / 16384.0 + W[:, None, None]
        assert np.abs(back - f).max() < 1e-15
        f_dev = torch.from_numpy(g.view(np.int16)).cuda()
        lbm.residual_sums_noalloc(desc, f_dev.data_ptr(), snap_u.data_ptr(), snap_v.data_ptr(), sums.data_ptr())
        torch.cuda.synchronize()
        got = sums.cpu().numpy()
        assert np.allclose(got, expected, rtol=1e-12, atol=1e-12), (got, expected)
        assert got[2] < case.cells - solid.sum() + 1.0  # solid cells are left out of sum rho


def test_noalloc_rejects_domains_beyond_the_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    desc = lbm.PopulationDesc(8192, 4096, 8192, lbm.STORAGE_F32, 0.5, 0.0, 0.0, None)
    assert 8192 * 4096 > lbm.NOALLOC_MAX_CELLS
    with pytest.raises(lbm.LbmError) as e:
        lbm.residual_sums_noalloc(desc, x.data_ptr(), x.data_ptr(), x.data_ptr(), x.data_ptr())
    assert e.value.status == lbm.ERR_INVALID
    assert "LBM_NOALLOC_MAX_CELLS" in str(e.value)
