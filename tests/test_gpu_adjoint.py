"""Differentiable SR-FMG: u = S(f) with the backward pass dL/df = S(dL/du)
(a second solve; A is symmetric, so this is the adjoint of the exact discrete
solve A^-1).

S is linear but not symmetric (the cycle is not), so the exact derivative of
the algorithm, S^T g, differs from S g by the order of the algebraic error.
Checks:
  - the backward pass equals the oracle's gradient (oracle solve of
    u - u_target, u from the oracle's forward) at 1e-11;
  - central finite differences of the quadratic loss equal <g, S d> (exact for
    a linear map, up to rounding) on 20 random directions;
  - the measured gap between <S g, d> and the finite differences (the
    cycle's asymmetry) stays below 1 % of the directional derivative, and
    the gradient is within 5 % of the exact discrete adjoint A^-1 (u - u_t).
"""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def loss_and_grad(gpu, solver, f, u_target):
    import torch
    ft = T(f).requires_grad_(True)
    u = gpu.solve_autograd(ft, solver)
    loss = 0.5 * ((u - T(u_target)) ** 2).sum()
    loss.backward()
    return float(loss), ft.grad.cpu().numpy(), u.detach().cpu().numpy()


@pytest.mark.parametrize("n,kw", [(32, dict(seg=16, K=2, A=4, B=0)),
                                  (64, dict(seg=16, K=2, A=8, B=0))])
def test_gradient_matches_oracle(gpu, oracle_mod, n, kw):
    f, _ = inputs.manufactured(n, 0)
    ut = inputs.target(n)
    with gpu.Solver(n, **kw) as s:
        _, grad, u = loss_and_grad(gpu, s, f, ut)
    u_or = oracle_mod.solve(f, **kw)
    g_or = oracle_mod.solve(u_or - ut, **kw)
    assert np.abs(u - u_or).max() <= 1e-11 * np.abs(u_or).max()
    assert np.abs(grad - g_or).max() <= 1e-11 * np.abs(g_or).max()


def test_gradient_matches_oracle_256(gpu, oracle_mod):
    """The differentiable configuration at full size: 256^3, 32^3 segments."""
    n = 256
    kw = dict(seg=32, K=3, A=8, B=0)
    f, _ = inputs.manufactured(n, 0)
    ut = inputs.target(n)
    with gpu.Solver(n, **kw) as s:
        _, grad, u = loss_and_grad(gpu, s, f, ut)
    u_or = oracle_mod.solve(f, **kw)
    g_or = oracle_mod.solve(u_or - ut, **kw)
    assert np.abs(grad - g_or).max() <= 1e-11 * np.abs(g_or).max()


def _fd_study(gpu, n, kw, directions=20):
    import torch
    f, _ = inputs.manufactured(n, 0)
    ut = inputs.target(n)
    rng = np.random.default_rng(3)
    out = []
    with gpu.Solver(n, **kw) as s:
        _, grad, u = loss_and_grad(gpu, s, f, ut)
        g = u - ut

        def loss(x):
            v = s.solve(T(x)).cpu().numpy()
            return 0.5 * float(((v - ut) ** 2).sum())

        for _ in range(directions):
            d = inputs.random_direction(n, rng)
            eps = 1e-2 * np.abs(f).max() / np.abs(d).max()
            fd = (loss(f + eps * d) - loss(f - eps * d)) / (2.0 * eps)
            Sd = s.solve(T(d)).cpu().numpy()
            out.append((fd, float(np.vdot(g, Sd)), float(np.vdot(grad, d))))
    return np.array(out)


def test_finite_differences(gpu):
    r = _fd_study(gpu, 32, dict(seg=16, K=2, A=4, B=0))
    fd, exact_adj, ad = r[:, 0], r[:, 1], r[:, 2]
    # central differences of a quadratic are exact: FD = <g, S d> = <S^T g, d>
    assert np.all(np.abs(fd - exact_adj) <= 1e-8 * np.abs(fd).max())
    # S g against S^T g: the asymmetry of the cycle, measured bound
    gap = np.abs(ad - fd).max() / np.abs(fd).max()
    assert gap < 0.01


def test_gradient_close_to_exact_discrete_adjoint(gpu):
    """dL/df of the exact discrete solve is A^-1 (u - u_target); the backward
    pass differs from it by the solver's algebraic error on u - u_target."""
    import exact
    n = 32
    kw = dict(seg=16, K=2, A=4, B=0)
    f, _ = inputs.manufactured(n, 0)
    ut = inputs.target(n)
    with gpu.Solver(n, **kw) as s:
        _, grad, u = loss_and_grad(gpu, s, f, ut)
    g_exact = exact.dst_solve(u - ut)
    assert np.abs(grad - g_exact).max() < 0.05 * np.abs(g_exact).max()
