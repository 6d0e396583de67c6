"""Parity of the iterative V-cycle solver (the comparison solver of Sec. 5.3,
Fig. "Errors of all solvers") through the C ABI with the oracle: same cycle
count, same final iterate to 1e-11, same relative residual; its argument
rules; and the figure's point on GB300-sized grids (error stagnation at a
fixed relative residual of 1e-4, FMG still second order)."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-11


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.mark.parametrize("n,rtol", [(2, 1e-4), (8, 1e-4), (16, 1e-4), (32, 1e-4), (48, 1e-6),
                                    (64, 1e-4), (128, 1e-4), (32, 1e-10)])
def test_vsolve_parity(gpu, oracle_mod, n, rtol):
    f, _ = inputs.manufactured(n, 1)
    ur, cr, qr = oracle_mod.vsolve(f, rtol=rtol)
    with gpu.Solver(n) as s:
        u, c, q = s.vsolve(T(f), rtol=rtol)
    u = u.cpu().numpy()
    assert c == cr
    assert np.abs(u - ur).max() <= TOL * np.abs(ur).max()
    # residual of the iterate difference the line above allows: |A| <= 12 n^2
    slack = 12.0 * n * n * TOL * np.abs(ur).max() / np.abs(f).max()
    assert q == pytest.approx(qr, rel=1e-6, abs=slack)


def test_vsolve_warm_start_and_limits(gpu, oracle_mod):
    n = 32
    f, _ = inputs.manufactured(n, 2)
    u0 = oracle_mod.solve(f)  # an FMG start
    ur, cr, qr = oracle_mod.vsolve(f, u0=u0, rtol=1e-8)
    with gpu.Solver(n) as s:
        u, c, q = s.vsolve(T(f), u=T(u0), rtol=1e-8)
        assert c == cr and np.abs(u.cpu().numpy() - ur).max() <= TOL * np.abs(ur).max()
        u, c, q = s.vsolve(T(f), max_cycles=0)
        assert c == 0 and q == 1.0 and not u.any()
        u, c, q = s.vsolve(T(f), rtol=1e-14, max_cycles=3)
        assert c == 3 and q > 1e-14
        u, c, q = s.vsolve(T(np.zeros_like(f)))
        assert c == 0 and q == 0.0


def test_vsolve_argument_rules(gpu):
    n = 32
    f, _ = inputs.manufactured(n, 0)
    with gpu.Solver(n, seg=16, K=1) as s:  # SR handle
        with pytest.raises(gpu.SRFMGError):
            s.vsolve(T(f))
    with gpu.Solver(n, mixed=True) as s:
        with pytest.raises(gpu.SRFMGError):
            s.vsolve(T(f))
    with gpu.Solver(n) as s:
        with pytest.raises(gpu.SRFMGError):
            s.vsolve(T(f), rtol=-1.0)
        bad = f.copy()
        bad[1, 2, 3] = np.inf
        with pytest.raises(gpu.SRFMGError) as e:
            s.vsolve(T(bad))
        assert e.value.status == gpu.SR_ERR_NONFINITE
        _, c, q = s.vsolve(T(f))  # the handle stays usable
        assert q <= 1e-4


def test_vsolve_error_stagnates(gpu):
    """At rtol = 1e-4 the V-cycle solver's error no longer falls from 256^3
    to 512^3 while FMG's error falls at second order."""
    ev, ef = {}, {}
    for n in (256, 512):
        f, uex = inputs.manufactured(n, 0)
        fd = T(f)
        with gpu.Solver(n) as s:
            u, c, q = s.vsolve(fd, rtol=1e-4)
            assert q <= 1e-4 and c <= 7
            ev[n] = np.abs(u.cpu().numpy() - uex).max()
            ef[n] = np.abs(s.solve(fd).cpu().numpy() - uex).max()
        del fd
    assert ef[256] / ef[512] > 3.0
    assert ev[256] / ev[512] < 1.5
