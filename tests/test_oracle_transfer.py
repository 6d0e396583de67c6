"""Pins for restriction (8-child average) and cell-centred trilinear
prolongation (Sec. 5.1: piecewise constant restriction, linear prolongation)."""
import numpy as np
import pytest

import exact


@pytest.mark.parametrize("n", [4, 8, 12])
def test_restriction_of_modes(oracle_mod, n):
    """avg of sin(w x) over x = X -+ h/2 is sin(w X) cos(w h / 2): a fine DST
    mode restricts to the coarse samples of the same sine times prod cos(k pi / 2n)."""
    rng = np.random.default_rng(n)
    for _ in range(5):
        k = tuple(int(v) for v in rng.integers(1, n + 1, size=3))
        fine = exact.mode(n, k)
        coarse = exact.mode(n // 2, k)
        fac = np.prod([np.cos(kd * np.pi / (2.0 * n)) for kd in k])
        assert np.allclose(oracle_mod.restrict(fine), fac * coarse, rtol=0, atol=1e-14)


def test_restriction_preserves_constants_and_means(oracle_mod):
    rng = np.random.default_rng(0)
    a = rng.standard_normal((8, 8, 8))
    r = oracle_mod.restrict(a)
    assert np.allclose(oracle_mod.restrict(np.full((6, 6, 6), 2.5)), 2.5)
    assert abs(r.mean() - a.mean()) < 1e-15
    assert abs(r[1, 2, 3] - a[2:4, 4:6, 6:8].mean()) < 1e-15


def _affine(n, c):
    x = (np.arange(n) + 0.5) / n
    return (c[0] + c[1] * x[None, None, :] + c[2] * x[None, :, None] + c[3] * x[:, None, None]
            + 0 * x[:, None, None])


@pytest.mark.parametrize("nc", [3, 4, 8])
def test_prolongation_reproduces_affine_fields_inside(oracle_mod, nc):
    c = (0.3, -1.2, 0.7, 2.1)
    fine = oracle_mod.prolong(_affine(nc, c))
    ref = _affine(2 * nc, c)
    s = slice(1, 2 * nc - 1)
    assert np.allclose(fine[s, s, s], ref[s, s, s], rtol=0, atol=1e-14)


def test_prolongation_boundary_cells(oracle_mod):
    """ghost = -mirror: a constant field gives 1/2 on fine face cells, 1/4 on
    edges and 1/8 in corners; a field linear through 0 at x = 0 is exact there."""
    nc = 4
    f = oracle_mod.prolong(np.ones((nc,) * 3))
    n = 2 * nc
    assert abs(f[0, 0, 0] - 0.125) < 1e-15
    assert abs(f[n // 2, n // 2, 0] - 0.5) < 1e-15
    assert abs(f[n // 2, 0, 0] - 0.25) < 1e-15
    assert abs(f[n // 2, n // 2, n // 2] - 1.0) < 1e-15
    X = (np.arange(nc) + 0.5) / nc
    g = oracle_mod.prolong(np.broadcast_to(X[None, None, :], (nc,) * 3).copy())
    x = (np.arange(n) + 0.5) / n
    assert np.allclose(g[n // 2, n // 2, : n // 2], x[: n // 2], atol=1e-15)


def test_prolongation_weights_sum_to_one(oracle_mod):
    rng = np.random.default_rng(5)
    a = rng.standard_normal((4, 4, 4))
    f = oracle_mod.prolong(a)
    # fine cells (2i+1, 2j+1, 2k+1) with i, j, k < 3 use coarse cells i..i+1 etc.
    w = np.array([0.75, 0.25])
    ref = np.einsum("a,b,c,cba->", w, w, w, a[1:3, 1:3, 1:3])
    assert abs(f[3, 3, 3] - ref) < 1e-14
