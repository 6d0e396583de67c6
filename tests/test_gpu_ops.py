"""Step-by-step parity of the CUDA kernels with the oracle's components, on
whole grids, through the C ABI (sr_op_*).  Sizes span several thread blocks
and ragged edges; FP64 tolerance 1e-11 relative max-norm (the bound the
whole solve is held to)."""
import numpy as np
import pytest

import exact

pytestmark = pytest.mark.gpu
TOL = 1e-11


def rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def N(t):
    return t.cpu().numpy()


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 33, 64])
def test_apply(gpu, oracle_mod, n):
    u = np.random.default_rng(n).standard_normal((n, n, n))
    assert rel(N(gpu.op_apply(T(u))), oracle_mod.apply(u)) < TOL


@pytest.mark.parametrize("n", [3, 16, 37])
def test_residual(gpu, oracle_mod, n):
    rng = np.random.default_rng(n)
    u, f = rng.standard_normal((2, n, n, n))
    assert rel(N(gpu.op_residual(T(u), T(f))), oracle_mod.residual(u, f)) < TOL


@pytest.mark.parametrize("nu", [1, 2, 3, 4])
@pytest.mark.parametrize("n", [4, 17, 48])
def test_smooth(gpu, oracle_mod, n, nu):
    rng = np.random.default_rng(10 * n + nu)
    u, f = rng.standard_normal((2, n, n, n))
    for lo, hi in [(1.0 / 6.0, 1.0), (0.1, 1.1)]:
        ref = oracle_mod.smooth(u, f, nu, lo, hi)
        assert rel(N(gpu.op_smooth(T(u), T(f), nu, lo, hi)), ref) < TOL


def test_smooth_mode_factor(gpu):
    """Closed-form Chebyshev factor on an eigenmode, straight on the GPU."""
    n = 16
    for k in [(1, 1, 1), (3, 7, 2), (16, 16, 16), (8, 1, 12)]:
        m = exact.mode(n, k)
        lam = exact.eigenvalue(n, k) / (6.0 * n * n)
        out = N(gpu.op_smooth(T(m), T(np.zeros_like(m)), 2))
        assert np.abs(out - exact.chebyshev_factor(lam, 2, 1.0 / 6.0, 1.0) * m).max() < 1e-13


@pytest.mark.parametrize("n", [2, 6, 32, 66])
def test_restrict(gpu, oracle_mod, n):
    a = np.random.default_rng(n).standard_normal((n, n, n))
    assert rel(N(gpu.op_restrict(T(a))), oracle_mod.restrict(a)) < TOL


@pytest.mark.parametrize("nc", [1, 2, 3, 8, 21, 32])
def test_prolong(gpu, oracle_mod, nc):
    a = np.random.default_rng(nc).standard_normal((nc, nc, nc))
    assert rel(N(gpu.op_prolong(T(a))), oracle_mod.prolong(a)) < TOL


@pytest.mark.parametrize("n", [2, 3, 4, 8, 9, 12, 16])
def test_coarse_solve(gpu, oracle_mod, n):
    """Up to 8^3 the dense inverse, above it the separable sine-transform solve."""
    f = np.random.default_rng(n).standard_normal((n, n, n))
    assert rel(N(gpu.op_coarse_solve(T(f))), oracle_mod.coarse_solve(f)) < TOL


def test_coarse_solve_32(gpu, oracle_mod):
    """The separable solve at its largest size, 32^3: against the exact DST
    solution and through its residual (the oracle's operator)."""
    n = 32
    f = np.random.default_rng(5).standard_normal((n, n, n))
    u = N(gpu.op_coarse_solve(T(f)))
    assert rel(u, exact.dst_solve(f)) < TOL
    assert np.abs(oracle_mod.apply(u) - f).max() < 1e-10 * np.abs(f).max()


def test_coarse_solve_separable_rectangle(gpu, oracle_mod):
    """32 x 16 x 16 cells of [0,2] x [0,1]^2 with the 27-point operator: the
    separable solve on unequal axes against the oracle's banded Cholesky."""
    geo = dict(lengths=(2, 1, 1), stencil=27, weights=(14 / 30, 3 / 30, 1 / 30))
    f = np.random.default_rng(7).standard_normal((16, 16, 32))
    assert rel(N(gpu.op_coarse_solve(T(f), **geo)), oracle_mod.coarse_solve(f, **geo)) < TOL


@pytest.mark.parametrize("n,kw", [(16, {}), (24, {}), (64, {}), (64, dict(n_coarse=8)),
                                  (64, dict(n_coarse=16)), (32, dict(n_coarse=16)),
                                  (32, dict(nu1=3, nu2=1)), (32, dict(nu1=1, nu2=4))])
def test_vcycle(gpu, oracle_mod, n, kw):
    rng = np.random.default_rng(n)
    f, u = rng.standard_normal((2, n, n, n))
    ref = oracle_mod.vcycle(f, u, **kw)
    assert rel(N(gpu.op_vcycle(T(f), T(u), **kw)), ref) < TOL
