"""Failure detection and recovery without a GPU fault.

A bounded wait that runs out is reported to the host as a status and the
context stays usable: lbm_bounded_wait_selftest makes one thread wait, with the
step kernels' own bounded wait (2 s limit), on an mbarrier that nothing
completes; the kernel raises the context's device error flag and returns, the
call reports LBM_ERR_CUDA once and clears the flag, and the solver keeps
stepping in parity with the oracle.  A device allocation that fails (injected
on the host through the allocator hook) makes lbm_create return LBM_ERR_OOM
after releasing everything it had obtained."""
import ctypes

import numpy as np
import pytest

import oracle as orc
import workloads as wl
from paper_1806_10251_gb300 import lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_expired_bounded_wait_is_reported_and_the_context_survives():
    c = wl.random_cavity_state(96, 40, 0.5, Re=60.0, seed=3)
    g = lbm.solver_from_case(c)
    g.step(5)
    st, waited = g.bounded_wait_selftest()
    assert st == lbm.ERR_CUDA, st
    assert "bounded wait expired" in lbm.last_error()
    assert 1.9 < waited < 30.0, waited
    # reported once: the flag is cleared, the next calls succeed
    r, _ = g.residual()
    assert np.isfinite(r)
    g.step(5)
    o = orc.Domain(c.nx, c.ny, c.nu, c.gamma, c.sides)
    o.init_equilibrium(c.rho0, c.ux0, c.uy0)
    o.step(10)
    assert np.abs(g.populations() - o.pops()).max() < 2e-6
    assert g.kernel_launches == 10
    g.close()


def test_injected_allocation_failure_is_reported_and_released():
    import torch
    blocks, calls = {}, [0]

    def _alloc(nbytes, _user):
        calls[0] += 1
        if calls[0] > 3:  # the fourth and later requests fail
            return None
        t = torch.empty(int(nbytes), dtype=torch.uint8, device="cuda")
        blocks[t.data_ptr()] = t
        return t.data_ptr()

    def _free(ptr, _user):
        blocks.pop(int(ptr), None)

    a = lbm.Allocator(lbm._ALLOC_FN(_alloc), lbm._FREE_FN(_free), None)
    lbm.check(lbm.lib().lbm_set_allocator(ctypes.byref(a)))
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.Solver(64, 64, 0.05, 0.5, 0.1)
        assert e.value.status == lbm.ERR_OOM
        assert calls[0] > 3 and not blocks  # everything obtained was released
    finally:
        lbm.lib().lbm_set_allocator(None)
    g = lbm.Solver(64, 64, 0.05, 0.5, 0.1)
    g.step(3)
    r, _ = g.residual()
    assert np.isfinite(r)
    g.close()
