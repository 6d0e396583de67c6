"""Segment sharding with redundant coarse solves (Sec. 7), on one GPU: the
segments of one problem split among several handles (segment ranges), each
SR stage split at the transition level, the two transition-level arrays
summed over the handles between the halves.  Joined through the host (the
arrays copied out, summed on the CPU and copied back) or on the device,
the handles reproduce the single-handle solve bit for bit: every
transition-level cell has one owner, so the sum is exact, and every other
step runs the same kernels on the same values."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def sharded_solve(gpu, n, f, parts, through_host, **kw):
    import torch
    nsegs = gpu.segment_count(n, kw["seg"], kw.get("lengths", (1, 1, 1)))
    ranges = [gpu.segment_range(nsegs, r, parts) for r in range(parts)]
    solvers = [gpu.Solver(n, segments=rg, **kw) for rg in ranges]
    ft = T(f)
    u = torch.full(ft.shape, float("nan"), dtype=torch.float64, device="cuda")
    try:
        if through_host:
            K = solvers[0].K
            for k in range(1, K + 1):
                for s in solvers:
                    s.stage_down(ft, k)
                bufs = [s.stage_buffers() for s in solvers]
                host = [sum(b[i].cpu() for b in bufs) for i in range(2)]
                for b in bufs:
                    for i in range(2):
                        b[i].copy_(host[i])
                for s in solvers:
                    s.stage_up(ft, k, u)
        else:
            gpu.solve_staged(solvers, ft, u)
        for s in solvers:
            s.check()
    finally:
        for s in solvers:
            s.close()
    return u.cpu().numpy()


CASES = [
    (128, dict(seg=32, K=3, A=11, B=1, n_coarse=16), 2),
    (64, dict(seg=16, K=2, A=8, B=0), 3),
    (64, dict(seg=16, K=3, J=[2, 4, 8]), 5),                 # maximum buffer schedule
    (16, dict(seg=8, K=2, J=[4, 4], lengths=(2, 1, 1), stencil=27), 3),
    (64, dict(seg=32, K=2, A=4, B=1), 8),                    # one segment per handle
]


@pytest.mark.parametrize("through_host", [True, False])
@pytest.mark.parametrize("n,kw,parts", CASES)
def test_shards_reproduce_single_handle(gpu, oracle_mod, n, kw, parts, through_host):
    if "lengths" in kw:
        f, _ = inputs.paper_problem(n)
    else:
        f, _ = inputs.manufactured(n, 5)
    with gpu.Solver(n, **kw) as s:
        ref = s.solve(T(f)).cpu().numpy()
    u = sharded_solve(gpu, n, f, parts, through_host, **kw)
    assert not np.isnan(u).any()
    assert np.array_equal(u, ref)


def test_full_size_two_shards(gpu, oracle_mod):
    """The benchmark workload split between two handles of 256 segments."""
    n = 256
    kw = workloads.config(workloads.SR256)
    f, _ = inputs.manufactured(n, 0)
    u = sharded_solve(gpu, n, f, 2, False, **kw)
    ref = oracle_mod.solve(f, **kw)
    assert np.abs(u - ref).max() / np.abs(ref).max() < 1e-11
    with gpu.Solver(n, **kw) as s:
        assert np.array_equal(u, s.solve(T(f)).cpu().numpy())


def test_one_handle_staged_equals_solve(gpu):
    import torch
    n = 64
    kw = dict(seg=16, K=2, A=8, B=0)
    f, _ = inputs.manufactured(n, 6)
    ft = T(f)
    with gpu.Solver(n, **kw) as s:
        ref = s.solve(ft).cpu()
        u = torch.empty_like(ft)
        gpu.solve_staged([s], ft, u)
        s.check()
    assert torch.equal(u.cpu(), ref)


def test_segment_range_rules(gpu):
    n = 64
    kw = dict(seg=16, K=2)
    with gpu.Solver(n, segments=(0, 32), **kw) as s:
        with pytest.raises(gpu.SRFMGError) as e:   # whole solves need every segment
            s.solve(T(np.zeros((n, n, n))))
        assert e.value.status == gpu.SR_ERR_INVALID
    for bad in [dict(segments=(60, 8), **kw),                 # past the 64 segments
                dict(segments=(0, 8), mixed=True, **kw),      # float64 only
                dict(segments=(0, 8)),                        # plain FMG has no segments
                dict(segments=(-1, 4), **kw)]:
        with pytest.raises(gpu.SRFMGError) as e:
            gpu.Solver(n, **bad)
        assert e.value.status == gpu.SR_ERR_INVALID
    with gpu.Solver(n, mixed=True, **kw) as s:             # mixed handles: no stages
        with pytest.raises(gpu.SRFMGError):
            s.stage_down(T(np.zeros((n, n, n))), 1)
