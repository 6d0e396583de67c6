"""The global V-cycle as one persistent cooperative launch (float64, 7-point,
degree-2 smoothers): from the first global level of at most 64^3 cells down
to the coarsest grid, the passes run inside one launch whose blocks meet at
a grid barrier.  Every cell takes the separate kernels' operations in the
same order, so solves with the persistent cycle equal the solves without it
bit for bit (the separate kernels are held to the oracle by the parity
tests); its barrier waits are bounded and, made to run out, the solve
reports SR_ERR_TIMEOUT and the handle stays usable."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    (256, workloads.config(workloads.SR256)),                 # transition level 32^3, 16^3 separable
    (256, workloads.config(workloads.PLAIN256)),              # plain FMG: levels 256..64 separate
    (64, dict(seg=16, K=2, A=8, B=0)),                         # 2^3 coarsest (dense inverse)
    (96, dict(seg=24, K=3, A=6, B=0)),                         # 3^3 coarsest
    (128, dict(n_coarse=8)),
    (48, dict(n_coarse=12)),                                   # 12^3 separable
    (32, dict(seg=16, K=3, A=4, B=0, lengths=(2, 1, 1))),      # a rectangle
    (64, dict(n_coarse=16, lengths=(2, 1, 1))),                # a rectangle, 32x16x16 separable
    (64, dict(seg=16, K=2, A=8, B=0, graph=True)),             # captured as a graph
]


@pytest.mark.parametrize("n,kw", CASES)
def test_persistent_equals_separate_kernels(gpu, n, kw):
    f, _ = inputs.paper_problem(n) if "lengths" in kw else inputs.manufactured(n, 8)
    with gpu.Solver(n, **kw) as s:
        assert s.debug_persistent_vcycle(True)
        a = s.solve(T(f)).cpu().numpy()
        launches_p = s.launches_per_solve
        s.debug_persistent_vcycle(False)
        b = s.solve(T(f)).cpu().numpy()
        launches_s = s.launches_per_solve
    assert np.array_equal(a, b)
    assert launches_p < launches_s


def test_persistent_vsolve_equals_separate(gpu):
    import torch
    n = 64
    f = T(inputs.manufactured(n, 2)[0])
    with gpu.Solver(n, n_coarse=16) as s:
        u1, c1, r1 = s.vsolve(f, torch.zeros_like(f), rtol=1e-8)
        s.debug_persistent_vcycle(False)
        u2, c2, r2 = s.vsolve(f, torch.zeros_like(f), rtol=1e-8)
    assert c1 == c2 and r1 == r2
    assert torch.equal(u1, u2)


def test_persistent_barrier_timeout_reported(gpu):
    n = 32
    f, _ = inputs.manufactured(n, 4)
    with gpu.Solver(n, seg=8, K=2, A=4, B=0) as s:
        assert s.debug_persistent_vcycle(True)
        ref = s.solve(T(f)).cpu().numpy()
        s.debug_force_wait_timeout(True)
        with pytest.raises(gpu.SRFMGError) as e:
            s.solve(T(f))
        assert e.value.status == gpu.SR_ERR_TIMEOUT
        s.debug_force_wait_timeout(False)
        again = s.solve(T(f)).cpu().numpy()
    assert np.array_equal(again, ref)


def test_mixed_and_27_point_handles_keep_separate_kernels(gpu):
    with gpu.Solver(64, seg=16, K=2, mixed=True) as s:
        assert not s.debug_persistent_vcycle(True)
    with gpu.Solver(16, lengths=(2, 1, 1), stencil=27) as s:
        assert not s.debug_persistent_vcycle(True)
