"""Batched solves (one CUDA graph for many right-hand sides on grids of
different sizes and configurations) against individual solves through the C
ABI, plus the full 64-problem mixed-precision workload sampled against the
oracle's float64 defect-correction loop."""
import numpy as np
import pytest

import exact
from paper_1406_7808_gb300 import inputs, workloads

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


PROBLEMS = [
    (16, dict()), (24, dict(seg=12, K=2, A=2, B=0)), (32, dict(seg=8, K=2, A=4, B=0)),
    (48, dict(mixed=True)), (32, dict(seg=16, K=2, A=8, B=0, mixed=True)),
    (64, dict(seg=16, K=2, A=8, B=0)), (16, dict(mixed=True, n_outer=3)),
]


def test_batch_equals_individual_solves(gpu):
    import torch
    fs = [T(inputs.manufactured(n, 10 + i)[0]) for i, (n, _) in enumerate(PROBLEMS)]
    solvers = [gpu.Solver(n, **kw) for n, kw in PROBLEMS]
    ref = [s.solve(f).cpu().numpy() for s, f in zip(solvers, fs)]
    us = [torch.empty_like(f) for f in fs]
    with gpu.Batch(solvers) as b:
        for streams in (1, 3):
            b.set_streams(streams)
            for u in us:
                u.zero_()
            b.solve(fs, us)
            for u, r in zip(us, ref):
                assert np.array_equal(u.cpu().numpy(), r)
        branches, ms = b.autotune(fs, us)
        assert 1 <= branches <= len(PROBLEMS) and ms > 0
        b.solve(fs, us)
        for u, r in zip(us, ref):
            assert np.array_equal(u.cpu().numpy(), r)
    us2 = [torch.empty_like(f) for f in fs]
    gpu.solve_batched(solvers, fs, us2)
    for u, r in zip(us2, ref):
        assert np.array_equal(u.cpu().numpy(), r)
    for s in solvers:
        s.close()


@pytest.mark.parametrize("n,kw", [(64, dict(seg=16, K=2, A=8, B=0)),
                                  (96, dict(seg=24, K=3, A=6, B=0, mixed=True)),
                                  (64, dict(seg=32, K=3, A=11, B=1, n_coarse=8))])
def test_launch_shape_does_not_change_results(gpu, n, kw):
    """The launch shape (cells in z per column-kernel thread, cells per
    per-cell-kernel thread) is a pure performance choice: every shape gives
    the same bits, in a single solve and inside a batch graph, which
    re-captures when a handle's shape changes."""
    import torch
    f = T(inputs.manufactured(n, 7)[0])
    with gpu.Solver(n, **kw) as s:
        assert s.launch_shape == (16, 2)
        ref = s.solve(f).cpu().numpy()
        for shape in [(1, 1), (7, 3), (8, 1), (32, 4), (256, 16)]:
            s.set_launch_shape(*shape)
            assert s.launch_shape == shape
            assert np.array_equal(s.solve(f).cpu().numpy(), ref)
        u = torch.empty_like(f)
        with gpu.Batch([s]) as b:
            b.solve([f], [u])
            assert np.array_equal(u.cpu().numpy(), ref)
            s.set_launch_shape(8, 4)
            u.zero_()
            b.solve([f], [u])
            assert np.array_equal(u.cpu().numpy(), ref)
        with pytest.raises(gpu.SRFMGError):
            s.set_launch_shape(0, 2)


def test_batch_rejects_repeated_outputs(gpu):
    import torch
    s1, s2 = gpu.Solver(16), gpu.Solver(16)
    f = T(inputs.manufactured(16, 0)[0])
    u = torch.empty_like(f)
    with gpu.Batch([s1, s2]) as b:
        with pytest.raises(gpu.SRFMGError) as e:
            b.solve([f, f], [u, u])
        assert e.value.status == gpu.SR_ERR_INVALID
    with pytest.raises(gpu.SRFMGError):
        gpu.Batch([s1, s1]).solve([f, f], [u, torch.empty_like(f)])


def test_full_batch_workload(gpu, oracle_mod):
    """64 right-hand sides, 16 each of 64^3, 128^3, 192^3, 256^3, mixed
    precision, one graph launch; sampled problems checked against the
    oracle's float64 defect-correction loop (0.1 e_disc)."""
    import torch
    from paper_1406_7808_gb300 import autotune
    problems = workloads.batch_problems()
    solvers, choices = autotune.tuned_batch(problems)
    fs, us = [], []
    for n, seed in problems:
        fs.append(T(inputs.manufactured(n, seed)[0]))
        us.append(torch.empty((n, n, n), dtype=torch.float64, device="cuda"))
    with gpu.Batch(solvers) as b:
        b.autotune(fs, us)
        b.solve(fs, us)
    for i in (0, 1, 2):  # one problem of 64^3, 128^3 and 192^3
        n, seed = problems[i]
        f, uex = inputs.manufactured(n, seed)
        kw = workloads.config(choices[n][0])
        okw = {k: v for k, v in kw.items() if k not in ("mixed", "n_outer")}
        assert kw["n_coarse"] == (12 if n == 192 else 16)
        ref = oracle_mod.solve_refined(f, kw["n_outer"], **okw)
        e_disc = np.abs(exact.dst_solve(f) - uex).max()
        assert np.abs(us[i].cpu().numpy() - ref).max() <= 0.1 * e_disc
    for s in solvers:
        s.close()
