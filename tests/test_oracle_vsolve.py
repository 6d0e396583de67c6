"""Pins for the oracle's iterative V-cycle solver (the comparison solver of
Sec. 5.3: V-cycles to a relative residual of 1e-4, Fig. "Errors of all
solvers").

- with a tight tolerance it reaches the exact discrete solution (DST solve);
- the reported relative residual is ||f - A u||_inf / ||f||_inf recomputed
  with an independent numpy stencil (dense Kronecker matrix on small grids);
- the stopping rule: the cycle count is the first one that meets rtol, each
  cycle contracts the residual by less than Gamma = 0.25;
- degenerate cases: max_cycles = 0, f = 0, a start at the exact solution;
- the error of the V-cycle solve stagnates under grid refinement at fixed
  rtol while FMG's keeps falling at second order (the figure's point).
"""
import numpy as np
import pytest

import exact
from paper_1406_7808_gb300 import inputs


def rel_resid(f, u):
    n = f.shape[0]
    r = f.ravel() - exact.dense_matrix(n) @ u.ravel()
    return np.abs(r).max() / np.abs(f).max()


@pytest.mark.parametrize("n", [8, 16, 32])
def test_tight_tolerance_reaches_discrete_solution(oracle_mod, n):
    f, _ = inputs.manufactured(n, 0)
    uh = exact.dst_solve(f)
    u, cycles, rel = oracle_mod.vsolve(f, rtol=1e-13, max_cycles=60)
    assert rel <= 1e-13 and cycles < 40
    assert np.abs(u - uh).max() < 1e-11 * np.abs(uh).max()


@pytest.mark.parametrize("n", [8, 16])
def test_reported_residual_is_the_relative_residual(oracle_mod, n):
    f, _ = inputs.manufactured(n, 2)
    for rtol in (1e-2, 1e-4, 1e-6):
        u, cycles, rel = oracle_mod.vsolve(f, rtol=rtol)
        assert rel == pytest.approx(rel_resid(f, u), rel=1e-9)
        assert rel <= rtol


@pytest.mark.parametrize("n", [16, 32, 64])
def test_stopping_rule_and_contraction(oracle_mod, n):
    f, _ = inputs.manufactured(n, 1)
    u, cycles, rel = oracle_mod.vsolve(f, rtol=1e-4)
    assert rel <= 1e-4
    # Gamma < 0.25 per cycle bounds the count: 0.25^7 < 1e-4
    assert 1 <= cycles <= 7
    # one cycle fewer does not meet the tolerance
    _, c1, rel1 = oracle_mod.vsolve(f, rtol=1e-4, max_cycles=cycles - 1)
    assert c1 == cycles - 1 and rel1 > 1e-4
    assert rel / rel1 < 0.25


def test_degenerate_cases(oracle_mod):
    n = 16
    f, _ = inputs.manufactured(n, 0)
    u, c, rel = oracle_mod.vsolve(f, max_cycles=0)
    assert c == 0 and rel == 1.0 and not u.any()
    u, c, rel = oracle_mod.vsolve(np.zeros_like(f))
    assert c == 0 and rel == 0.0 and not u.any()
    uh = exact.dst_solve(f)
    u, c, rel = oracle_mod.vsolve(f, u0=uh, rtol=1e-8)
    assert c == 0 and rel < 1e-8 and np.array_equal(u, uh)
    with pytest.raises(RuntimeError):
        bad = f.copy()
        bad[3, 4, 5] = np.nan
        oracle_mod.vsolve(bad)


@pytest.mark.slow
def test_error_stagnates_under_refinement(oracle_mod):
    """Fig. "Errors of all solvers": at a fixed relative residual of 1e-4 the
    V-cycle solver's error stops falling with h while FMG's falls at second
    order (here: 128^3 -> 256^3, error ratio < 1 against > 3 for FMG)."""
    err_v, err_f = {}, {}
    for n in (128, 256):
        f, uex = inputs.manufactured(n, 0)
        u, cycles, rel = oracle_mod.vsolve(f, rtol=1e-4)
        err_v[n] = np.abs(u - uex).max()
        err_f[n] = np.abs(oracle_mod.solve(f) - uex).max()
    assert err_f[128] / err_f[256] > 3.0
    assert err_v[128] / err_v[256] < 1.0
