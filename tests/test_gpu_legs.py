"""Segment-resident legs of the float32 inner solver (SR_MIXED; a mode that
is off by default, the separate kernels being faster on GB300): on the SR
levels below each stage's top, one thread-block cluster per segment holds
the segment's box in shared memory for the down-leg's pre-smoother and
restriction and for the up-leg (correction, post-smoother, w - t).  They
compute every cell with the separate kernels' operations in the same order,
so a solve with the legs equals the solve without them bit for bit; the
separate kernels are in turn held to the float64 oracle loop by
tests/test_gpu_mixed.py.

The legs' device-side waits are bounded: made to run out (a debug switch
that has them expect data that never arrives), the solve reports
SR_ERR_TIMEOUT after about a second per wait and the handle stays usable."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    (128, dict(seg=32, K=3, A=8, B=0)),
    (128, dict(seg=32, K=3, A=11, B=1, n_coarse=16)),
    (256, dict(seg=64, K=4, A=8, B=0, n_coarse=16)),        # the 512^3 workload's boxes
    (96, dict(seg=24, K=3, A=6, B=0)),
    (64, dict(seg=16, K=3, J=[2, 4, 8])),                    # maximum buffer schedule
    (64, dict(seg=32, K=4, A=4, B=1)),                       # boxes clipped at the domain
    (32, dict(seg=16, K=3, A=4, B=0, lengths=(2, 1, 1))),    # a rectangle
    (128, dict(seg=32, K=3, A=8, B=0, graph=True)),          # captured as a graph
]


@pytest.mark.parametrize("n,kw", CASES)
def test_legs_equal_separate_kernels(gpu, n, kw):
    f, _ = (inputs.paper_problem(n) if "lengths" in kw else inputs.manufactured(n, 3))
    with gpu.Solver(n, mixed=True, n_outer=2, **kw) as s:
        levels = s.debug_segment_legs(True)
        assert levels, "no SR level qualified for a leg"
        a = s.solve(T(f)).cpu().numpy()
        s.debug_segment_legs(False)
        b = s.solve(T(f)).cpu().numpy()
        s.debug_segment_legs(True)
        c = s.solve(T(f)).cpu().numpy()
    assert np.isfinite(a).all()
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


def test_legs_cover_the_coarse_sr_levels(gpu):
    """The 512^3 workload's geometry (64^3 segments, K = 4): levels 1 to 3 of
    the SR hierarchy (boxes of 24^3, 32^3 and 48^3 cells) run as legs."""
    with gpu.Solver(256, seg=64, K=4, A=8, B=0, n_coarse=16, mixed=True) as s:
        assert s.debug_segment_legs(True) == [1, 2, 3]


def test_leg_wait_timeout_is_reported(gpu):
    n = 32
    kw = dict(seg=16, K=3, A=4, B=0, mixed=True, n_outer=1)
    f, _ = inputs.manufactured(n, 4)
    with gpu.Solver(n, **kw) as s:
        assert s.debug_segment_legs(True)
        ref = s.solve(T(f)).cpu().numpy()
        s.debug_force_wait_timeout(True)
        with pytest.raises(gpu.SRFMGError) as e:
            s.solve(T(f))
        assert e.value.status == gpu.SR_ERR_TIMEOUT
        s.debug_force_wait_timeout(False)
        again = s.solve(T(f)).cpu().numpy()
    assert np.array_equal(again, ref)
