"""sr_op_smooth_noalloc (the smoother with its scratch in a fixed device array,
for callers that cannot allocate device memory) against the allocating
sr_op_smooth, through the C ABI.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 1e-11


def _T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,nu", [(17, 2), (64, 2), (33, 3), (64, 1)])
def test_noalloc_matches_allocating_smoother_twice(gpu, n, nu):
    import torch
    rng = np.random.default_rng(100 + n + nu)
    for call in range(2):  # two calls in a row: the shared scratch keeps stale data
        u, f = rng.standard_normal((2, n, n, n))
        ref = gpu.op_smooth(_T(u), _T(f), nu).cpu().numpy()
        out = gpu.op_smooth_noalloc(_T(u), _T(f), nu)
        torch.cuda.synchronize()
        out = out.cpu().numpy()
        err = np.abs(out - ref).max() / np.abs(ref).max()
        assert err < TOL, (call, err)


def test_noalloc_rejects_sizes_above_the_maximum(gpu):
    import torch
    n = gpu.NOALLOC_MAX_N + 1
    u = torch.zeros((n, n, n), dtype=torch.float64, device="cuda")
    st = gpu.load().sr_op_smooth_noalloc(n, 2, 1.0 / 6.0, 1.0, ctypes.c_void_p(u.data_ptr()),
                                         ctypes.c_void_p(u.data_ptr()), None)
    assert st == gpu.SR_ERR_UNSUPPORTED_SIZE
