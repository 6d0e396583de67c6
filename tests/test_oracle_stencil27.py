"""Pins for the oracle on the paper's own model problem (Sec. 5.1): a
27-point operator on the rectangular domain [0, 2] x [0, 1] x [0, 1] with
4 x 2 x 2 cubic segments.

The paper names the stencil only as a "27-point finite volume stencil that
is 2nd-order accurate"; the operator here is the general reflection-
symmetric one, A u = n^2 (w0 u - w1 sum_faces - w2 sum_edges - w3 sum_corners)
with w1 + 4 w2 + 4 w3 = 1, tested with two readings: the finite-volume
stencil whose face fluxes are Simpson averages over the 3 x 3 transverse
cells (w = (0, 1/6, 1/12), which is also the trilinear finite-element
stiffness matrix) and the (14, 3, 1)/30 stencil.

- operator: equal to a Kronecker-product assembly, and diagonal on the
  discrete sine modes with the closed-form symbol, for cubes and rectangles;
- coarsest solve: equal to a dense direct solve;
- smoother: the Chebyshev factor on eigenmodes is T_nu in closed form with
  lambda_max taken from the symbol's corners;
- V-cycle: converges to the exact discrete solution (DST solve);
- FMG on the paper's u = prod (x_i^4 - R_i^2 x_i^2): second-order total
  error and an algebraic error well below the discretisation error
  ("asymptotically exact", Sec. 5.3);
- SR: equal to the independent masked implementation on rectangular
  segment layouts, and to plain FMG when buffers cover the whole level.
"""
import itertools

import numpy as np
import pytest

import exact
import sr_masked
from paper_1406_7808_gb300 import inputs

SIMPSON = (0.0, 1.0 / 6.0, 1.0 / 12.0)
W1430 = (14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)
WEIGHTS = [SIMPSON, W1430]
RECT = (2, 1, 1)


def geo(w, lengths=RECT):
    return dict(lengths=lengths, stencil=27, weights=w)


def shape_of(n, lengths):
    return (n * lengths[2], n * lengths[1], n * lengths[0])


@pytest.mark.parametrize("w", WEIGHTS + [(1.0, 0.0, 0.0)])
@pytest.mark.parametrize("lengths", [(1, 1, 1), (2, 1, 1), (1, 3, 2)])
def test_operator_against_kronecker_assembly(oracle_mod, w, lengths):
    n = 4
    shape = shape_of(n, lengths)
    u = np.random.default_rng(1).standard_normal(shape)
    A = exact.dense_matrix_g(shape, n, w)
    a = oracle_mod.apply(u, **geo(w, lengths))
    assert np.abs(a.ravel() - A @ u.ravel()).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("w", WEIGHTS)
def test_operator_eigenmodes(oracle_mod, w):
    n = 8
    shape = shape_of(n, RECT)
    for k in [(1, 1, 1), (16, 8, 8), (3, 5, 2), (16, 1, 7), (9, 8, 1)]:
        v = exact.mode_g(shape, k)
        lam = exact.eigenvalue_g(shape, n, w, k)
        Av = oracle_mod.apply(v, **geo(w))
        assert np.abs(Av - lam * v).max() <= 1e-12 * abs(lam)


def test_symbol_corner_values():
    """lambda_max(D^-1 A): 2 for the 7-point operator, 3/2 for the Simpson
    stencil (at one oscillating direction), 184/128 for (14, 3, 1)/30 (at
    the checkerboard)."""
    def lmax(w):
        w0 = 6 * w[0] + 12 * w[1] + 8 * w[2]
        return max(exact.symbol(w, c) for c in itertools.product((-1, 1), repeat=3)) / w0
    assert lmax((1.0, 0.0, 0.0)) == pytest.approx(2.0)
    assert lmax(SIMPSON) == pytest.approx(1.5)
    assert lmax(W1430) == pytest.approx(184.0 / 128.0)


@pytest.mark.parametrize("w", WEIGHTS)
@pytest.mark.parametrize("n,lengths", [(2, (2, 1, 1)), (3, (2, 1, 1)), (2, (1, 1, 1))])
def test_coarse_solve_is_direct_solve(oracle_mod, w, n, lengths):
    shape = shape_of(n, lengths)
    f = np.random.default_rng(2).standard_normal(shape)
    ud = np.linalg.solve(exact.dense_matrix_g(shape, n, w), f.ravel()).reshape(shape)
    u = oracle_mod.coarse_solve(f, **geo(w, lengths))
    assert np.abs(u - ud).max() <= 1e-12 * np.abs(ud).max()


@pytest.mark.parametrize("w", WEIGHTS)
@pytest.mark.parametrize("nu", [1, 2, 3])
def test_smoother_factor_on_eigenmodes(oracle_mod, w, nu):
    n = 8
    shape = shape_of(n, RECT)
    w0 = 6 * w[0] + 12 * w[1] + 8 * w[2]
    lmax = max(exact.symbol(w, c) for c in itertools.product((-1, 1), repeat=3)) / w0
    for k in [(1, 1, 1), (16, 8, 8), (10, 3, 6), (2, 8, 1)]:
        v = exact.mode_g(shape, k)
        lam = exact.eigenvalue_g(shape, n, w, k) / (w0 * n * n)  # of D^-1 A
        u = oracle_mod.smooth(v, np.zeros(shape), nu, **geo(w))
        expected = exact.chebyshev_factor(lam / lmax * 2.0, nu, 1.0 / 6.0, 1.0)
        assert np.abs(u - expected * v).max() <= 1e-12


@pytest.mark.parametrize("w", WEIGHTS)
def test_vcycle_converges_to_discrete_solution(oracle_mod, w):
    n = 8
    f, _ = inputs.paper_problem(n)
    uh = exact.dst_solve_g(f, n, w)
    u = np.zeros_like(f)
    errs = []
    for _ in range(25):
        u = oracle_mod.vcycle(f, u, **geo(w))
        errs.append(np.abs(u - uh).max())
    assert errs[-1] < 1e-11 * np.abs(uh).max()
    assert errs[6] / errs[5] < 0.25


@pytest.mark.parametrize("w", WEIGHTS)
def test_fmg_second_order_and_asymptotically_exact(oracle_mod, w):
    err, alg, disc = [], [], []
    for n in (8, 16, 32, 64):
        f, u = inputs.paper_problem(n)
        uf = oracle_mod.solve(f, **geo(w))
        uh = exact.dst_solve_g(f, n, w)
        err.append(np.abs(uf - u).max())
        alg.append(np.abs(uf - uh).max())
        disc.append(np.abs(uh - u).max())
    ratios = [err[i] / err[i + 1] for i in range(3)]
    assert all(3.6 < r < 4.4 for r in ratios), ratios
    assert all(a < 0.2 * d for a, d in zip(alg, disc))


GEOMS = [(8, 4, 1, [2]), (16, 8, 2, [2, 4]), (16, 8, 2, [4, 4]), (16, 4, 2, [2, 2]),
         (32, 16, 3, [4, 4, 4])]


@pytest.mark.parametrize("w", WEIGHTS)
@pytest.mark.parametrize("n,seg,K,J", GEOMS)
def test_sr_matches_masked_implementation(oracle_mod, w, n, seg, K, J):
    f, _ = inputs.paper_problem(n)
    a = oracle_mod.solve(f, seg=seg, K=K, J=J, **geo(w))
    b = sr_masked.sr_fmg(f, seg, K, J, sr_masked.Params(**geo(w)))
    assert not np.isnan(b).any()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_sr_masked_seven_point_rectangle(oracle_mod):
    n, seg, K, J = 16, 8, 2, [2, 4]
    f, _ = inputs.paper_problem(n)
    g = dict(lengths=RECT)
    a = oracle_mod.solve(f, seg=seg, K=K, J=J, **g)
    b = sr_masked.sr_fmg(f, seg, K, J, sr_masked.Params(lengths=RECT))
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


@pytest.mark.parametrize("w", WEIGHTS)
def test_whole_level_buffers_are_plain_fmg(oracle_mod, w):
    n, seg, K = 16, 8, 2
    f, _ = inputs.paper_problem(n)
    J = [2 * n >> (K - k) for k in range(1, K + 1)]  # beyond the longest side
    a = oracle_mod.solve(f, seg=seg, K=K, J=J, **geo(w))
    b = oracle_mod.solve(f, **geo(w))
    assert np.array_equal(a, b)


def test_rejects_bad_operators_and_layouts(oracle_mod):
    ok = dict(n=16, seg=8, K=2, J=[2, 4], lengths=RECT, stencil=27)
    assert oracle_mod.check_config(weights=SIMPSON, **ok) == 0
    assert oracle_mod.check_config(weights=(0.5, 0.1, 0.1), **ok) != 0   # inconsistent
    assert oracle_mod.check_config(weights=(-1.0, 0.25, 0.25), **ok) != 0  # not definite
    assert oracle_mod.check_config(weights=SIMPSON, **dict(ok, stencil=9)) != 0
    assert oracle_mod.check_config(weights=SIMPSON, **dict(ok, seg=12)) != 0
