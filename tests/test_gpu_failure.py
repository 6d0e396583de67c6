"""Failure paths of the C ABI on the GPU, made on the host (nothing here
faults or hangs the device).

Allocation failure: sr_debug_fail_alloc makes the k-th device allocation
fail as out of memory.  Sweeping k over every allocation of sr_fmg_create
(float64 SR, mixed precision, the separable coarsest solve, the 27-point
operator), each create must return SR_ERR_OOM with a NULL handle and leave
no device memory held by the library (its own count of live bytes is back
where it was, and the device's free memory has not drifted); the library
then still solves correctly.  The pipelined host path's staging allocation
fails the same way without spoiling the handle."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu

CREATE_CASES = [
    (64, dict(seg=16, K=2)),
    (64, dict(seg=16, K=2, mixed=True)),
    (32, dict(n_coarse=16)),
    (16, dict(seg=8, K=2, J=[4, 4], lengths=(2, 1, 1), stencil=27)),
]


@pytest.mark.parametrize("n,kw", CREATE_CASES)
def test_create_allocation_failure_is_oom_without_leak(gpu, n, kw):
    import torch
    c0 = gpu.debug_alloc_count()
    with gpu.Solver(n, **kw):
        pass
    total = gpu.debug_alloc_count() - c0
    assert total > 3
    live0 = gpu.debug_live_bytes()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    try:
        for k in range(1, total + 1):
            gpu.debug_fail_alloc(k)
            with pytest.raises(gpu.SRFMGError) as e:
                gpu.Solver(n, **kw)
            assert e.value.status == gpu.SR_ERR_OOM
            assert gpu.debug_live_bytes() == live0
    finally:
        gpu.debug_fail_alloc(0)
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) <= 4 << 20
    f, _ = inputs.manufactured(n, 0) if "lengths" not in kw else inputs.paper_problem(n)
    with gpu.Solver(n, **kw) as s:
        u = s.solve(torch.from_numpy(f).cuda()).cpu().numpy()
    assert np.isfinite(u).all()


def test_host_staging_allocation_failure(gpu):
    import torch
    n = 32
    f, _ = inputs.manufactured(n, 0)
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    with gpu.Solver(n, seg=8, K=2) as s:
        ref = s.solve(torch.from_numpy(f).cuda()).cpu()
        gpu.debug_fail_alloc(1)
        try:
            with pytest.raises(gpu.SRFMGError) as e:
                s.solve_host_async(fh, uh)
            assert e.value.status == gpu.SR_ERR_OOM
        finally:
            gpu.debug_fail_alloc(0)
        s.solve_host_async(fh, uh)
        s.check_host()
        assert torch.equal(uh, ref)


def test_injection_argument_checked(gpu):
    with pytest.raises(gpu.SRFMGError) as e:
        gpu.debug_fail_alloc(-1)
    assert e.value.status == gpu.SR_ERR_INVALID
