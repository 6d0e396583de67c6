"""Graph mode (sr_fmg_config.graph = 1): each solve is queued as one captured
CUDA graph.  The graph holds the same kernels in the same order, so results
must be bit-identical to kernel-by-kernel solves; a new (f, u) pair is
recaptured; the status of a solve (a non-finite f) still reaches
sr_fmg_check; the per-kernel profiler falls back to kernel-by-kernel
launches."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [(64, dict(seg=16, K=2, A=8, B=0)), (64, {}), (64, dict(seg=32, K=2, mixed=True)),
         (32, dict(seg=16, K=2, J=[4, 4], lengths=(2, 1, 1), stencil=27))]


@pytest.mark.parametrize("n,kw", CASES)
def test_graph_matches_direct(gpu, n, kw):
    import torch
    lengths = kw.get("lengths", (1, 1, 1))
    sh = gpu.grid_shape(n, lengths)
    f1 = inputs.paper_problem(n, lengths=lengths, R=lengths)[0] if lengths != (1, 1, 1) else \
        inputs.manufactured(n, 1)[0]
    f2 = 0.5 * f1 + 1.0
    with gpu.Solver(n, **kw) as d, gpu.Solver(n, graph=True, **kw) as g:
        a = d.solve(T(f1)).cpu().numpy()
        b = d.solve(T(f2)).cpu().numpy()
        ft1, ft2 = T(f1), T(f2)
        u = torch.empty(sh, dtype=torch.float64, device="cuda")
        for _ in range(3):  # capture once, then relaunch
            g.solve(ft1, u)
            assert np.array_equal(u.cpu().numpy(), a)
        g.solve(ft2, u)  # new pair: recapture
        assert np.array_equal(u.cpu().numpy(), b)
        g.solve(ft1, u)
        assert np.array_equal(u.cpu().numpy(), a)
        assert np.array_equal(g.solve_host(f2), b)
        assert g.launches_per_solve == d.launches_per_solve


def test_graph_reports_status(gpu):
    n = 32
    f, _ = inputs.manufactured(n, 0)
    with gpu.Solver(n, seg=16, K=2, graph=True) as g:
        ft = T(f)
        u = g.solve(ft)
        bad = ft.clone()
        bad[1, 2, 3] = float("nan")
        with pytest.raises(gpu.SRFMGError) as e:
            g.solve(bad)
        assert e.value.status == gpu.SR_ERR_NONFINITE
        assert np.array_equal(g.solve(ft).cpu().numpy(), u.cpu().numpy())


def test_graph_mode_profiles_kernel_by_kernel(gpu):
    n = 64
    f, _ = inputs.manufactured(n, 0)
    with gpu.Solver(n, seg=32, K=2, graph=True) as g:
        ft = T(f)
        ref = g.solve(ft).cpu().numpy()
        g.profile(True)
        u = g.solve(ft)
        prof = g.profile_read()
        g.profile(False)
        assert sum(v["launches"] for v in prof.values()) == g.launches_per_solve
        assert np.array_equal(u.cpu().numpy(), ref)


@pytest.mark.parametrize("kw", [dict(seg=16, K=2, A=8, B=0, graph=True), dict(mixed=True)])
def test_pipelined_host_solves(gpu, kw):
    """sr_fmg_solve_host_async: a run of solves from host arrays with copies
    overlapping the neighbouring solves gives each f the same u as the
    synchronous host solve; a non-finite f in the run is reported by
    sr_fmg_check_host and the handle stays usable."""
    import torch
    n = 64
    fs = [torch.from_numpy(inputs.manufactured(n, s)[0]).pin_memory() for s in range(5)]
    outs = [torch.empty_like(f).pin_memory() for f in fs]
    with gpu.Solver(n, **kw) as s:
        ref = [s.solve_host(f.numpy()) for f in fs]
        for f, o in zip(fs, outs):
            s.solve_host_async(f, o)
        s.check_host()
        for r, o in zip(ref, outs):
            assert np.array_equal(r, o.numpy())
        bad = fs[2].clone()
        bad[1, 2, 3] = float("nan")
        s.solve_host_async(fs[0], outs[0])
        s.solve_host_async(bad, outs[1])
        s.solve_host_async(fs[1], outs[2])
        with pytest.raises(gpu.SRFMGError) as e:
            s.check_host()
        assert e.value.status == gpu.SR_ERR_NONFINITE
        s.solve_host_async(fs[3], outs[3])
        s.check_host()
        assert np.array_equal(outs[3].numpy(), ref[3])
