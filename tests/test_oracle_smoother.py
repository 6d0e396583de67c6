"""Pins for the Chebyshev smoother (Sec. 5.1: degree-2 pre/post smoothers,
degree-1 before each FMG V-cycle): on an eigenmode of D^-1 A with f = 0 the
smoother multiplies the mode by the Chebyshev factor p_nu(lambda), evaluated
here in closed form (cos / cosh of nu times arccos / arccosh)."""
import numpy as np
import pytest

import exact


@pytest.mark.parametrize("nu", [1, 2, 3])
@pytest.mark.parametrize("interval", [(1.0 / 6.0, 1.0), (0.1, 1.1), (0.05, 1.0)])
def test_chebyshev_mode_factor(oracle_mod, nu, interval):
    n = 8
    rng = np.random.default_rng(nu)
    for _ in range(4):
        k = tuple(int(v) for v in rng.integers(1, n + 1, size=3))
        m = exact.mode(n, k)
        lam = exact.eigenvalue(n, k) / (6.0 * n * n)  # eigenvalue of D^-1 A
        out = oracle_mod.smooth(m, np.zeros_like(m), nu, *interval)
        fac = exact.chebyshev_factor(lam, nu, *interval)
        assert np.allclose(out, fac * m, rtol=0, atol=1e-13)


def test_degree_one_is_damped_jacobi(oracle_mod):
    rng = np.random.default_rng(2)
    n = 6
    u, f = rng.standard_normal((2, n, n, n))
    lo, hi = 1.0 / 6.0, 1.0
    omega = 1.0 / (lo + hi)  # 1 / theta with theta = (2 lo + 2 hi) / 2
    r = f - (exact.dense_matrix(n) @ u.ravel()).reshape(n, n, n)
    ref = u + omega * r / (6.0 * n * n)
    assert np.allclose(oracle_mod.smooth(u, f, 1, lo, hi), ref, rtol=0, atol=1e-13)


def test_smoother_fixed_point(oracle_mod):
    n = 8
    rng = np.random.default_rng(4)
    f = rng.standard_normal((n, n, n))
    uh = exact.dst_solve(f)
    assert np.allclose(oracle_mod.smooth(uh, f, 2), uh, rtol=0, atol=1e-14 * np.abs(uh).max() * 10)


@pytest.mark.parametrize("geo", [{}, dict(lengths=(2, 1, 1), stencil=27)])
def test_first_coarse_smoother_step_from_restricted_residual(oracle_mod, geo):
    """After restriction (Sec. 2, FAS cycle: u_c = I u, rhs_c = rho + A_c u_c)
    the coarse smoother's first residual f - A u is rho itself, so a degree-2
    pass from (u_c, rhs_c) equals the same pass from (u_c, rho + A_c u_c)
    whatever order the terms are formed in; the float64 GPU path relies on
    this to take the first residual D^-1 rho from the coarse right-hand-side
    pass.  Checked on the oracle's own residual, restriction and smoother."""
    rng = np.random.default_rng(7)
    lengths = geo.get("lengths", (1, 1, 1))
    n = 16
    shape = (n * lengths[2], n * lengths[1], n * lengths[0])
    u = rng.standard_normal(shape)
    f = rng.standard_normal(shape) * n * n
    rho = oracle_mod.restrict(oracle_mod.residual(u, f, **geo), **geo)
    uc = oracle_mod.restrict(u, **geo)
    rhs = rho + oracle_mod.apply(uc, **geo)
    first = oracle_mod.residual(uc, rhs, **geo)
    scale = np.abs(rhs).max()
    assert np.abs(first - rho).max() <= 1e-13 * scale
    # two different roundings of the same right-hand side smooth to the same u
    a = oracle_mod.smooth(uc, rhs, 2, **geo)
    b = oracle_mod.smooth(uc, rho + (rhs - rho), 2, **geo)
    assert np.abs(a - b).max() <= 1e-13 * max(1.0, np.abs(a).max())


@pytest.mark.parametrize("interval", [(1.0 / 6.0, 1.0), (0.1, 1.1)])
def test_fused_fmg_step_residual(oracle_mod, interval):
    """The degree-1 step u1 = u + beta r (r = D^-1 (f - A u), beta = 1/theta
    of the Chebyshev interval, Sec. 5.1 smoother) leaves the residual
    D^-1 (f - A u1) = r - beta D^-1 A r = (1 - beta) r + (beta/6) S(r),
    S the 7-point neighbour sum with the boundary ghosts of A; the FMG step
    kernel forms the next smoother's first residual this way.  Checked on the
    oracle's own smoother and operator, with S(r) = 6 r - A r / n^2."""
    rng = np.random.default_rng(11)
    n = 12
    u = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n)) * n * n
    lo, hi = interval
    beta = 1.0 / (lo + hi)  # 1 / theta, lambda_max(D^-1 A) = 2
    d = 6.0 * n * n
    r = oracle_mod.residual(u, f) / d
    u1 = oracle_mod.smooth(u, f, 1, lo, hi)
    assert np.allclose(u1, u + beta * r, rtol=0, atol=1e-13 * np.abs(u).max())
    literal = oracle_mod.residual(u1, f) / d
    s = 6.0 * r - oracle_mod.apply(r) / (n * n)
    fused = (1.0 - beta) * r + (beta / 6.0) * s
    assert np.abs(literal - fused).max() <= 1e-12 * np.abs(r).max()
