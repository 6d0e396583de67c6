"""Pins for the oracle's operator, boundary condition and coarsest solve.

The 7-point operator with ghost = -mirror (Sec. 2, Eq. eq:deq; Sec. 3.3) is
diagonalised by DST-II modes with closed-form eigenvalues; a dropped
neighbour, a wrong ghost sign or a wrong h scaling breaks the eigen-relation.
"""
import numpy as np
import pytest

import exact


@pytest.mark.parametrize("n", [2, 3, 4, 5, 8, 12])
def test_operator_eigenmodes(oracle_mod, n):
    rng = np.random.default_rng(n)
    for _ in range(6):
        k = tuple(int(v) for v in rng.integers(1, n + 1, size=3))
        m = exact.mode(n, k)
        out = oracle_mod.apply(m)
        lam = exact.eigenvalue(n, k)
        assert np.allclose(out, lam * m, rtol=0, atol=1e-11 * lam * max(1.0, np.abs(m).max()))


def test_operator_symmetric(oracle_mod):
    rng = np.random.default_rng(1)
    n = 7
    x, y = rng.standard_normal((2, n, n, n))
    lhs = np.vdot(oracle_mod.apply(x), y)
    rhs = np.vdot(x, oracle_mod.apply(y))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("n", [2, 3, 4])
def test_operator_matches_kronecker_matrix(oracle_mod, n):
    """Columns of the oracle operator equal the Kronecker-sum matrix, itself
    pinned by its DST eigen-decomposition below."""
    M = exact.dense_matrix(n)
    cols = []
    for q in range(n ** 3):
        e = np.zeros(n ** 3)
        e[q] = 1.0
        cols.append(oracle_mod.apply(e.reshape(n, n, n)).ravel())
    assert np.allclose(np.array(cols).T, M, rtol=0, atol=1e-12 * n * n)


@pytest.mark.parametrize("n", [4, 8])
def test_kronecker_matrix_eigenvalues(n):
    M = exact.dense_matrix(n)
    ev = np.sort(np.linalg.eigvalsh(M))
    L1 = exact.lam1(n)
    ref = np.sort((L1[:, None, None] + L1[None, :, None] + L1[None, None, :]).ravel())
    assert np.allclose(ev, ref, rtol=1e-12)


@pytest.mark.parametrize("n", [2, 3])
def test_coarse_solve_is_exact(oracle_mod, n):
    rng = np.random.default_rng(10 + n)
    f = rng.standard_normal((n, n, n))
    u = oracle_mod.coarse_solve(f)
    assert np.allclose(u, exact.dst_solve(f), rtol=0, atol=1e-13 * np.abs(u).max())
    assert np.allclose(exact.dense_matrix(n) @ u.ravel(), f.ravel(), atol=1e-12 * np.abs(f).max())


@pytest.mark.parametrize("n", [4, 8])
def test_dst_solve_equals_dense_solve(n):
    """The exact solver used as a reference elsewhere equals the direct dense solve."""
    rng = np.random.default_rng(n)
    f = rng.standard_normal((n, n, n))
    ud = np.linalg.solve(exact.dense_matrix(n), f.ravel()).reshape(n, n, n)
    assert np.allclose(exact.dst_solve(f), ud, rtol=0, atol=1e-14 * np.abs(ud).max() * n)


def test_residual(oracle_mod):
    rng = np.random.default_rng(3)
    n = 6
    u, f = rng.standard_normal((2, n, n, n))
    r = oracle_mod.residual(u, f)
    ref = f - (exact.dense_matrix(n) @ u.ravel()).reshape(n, n, n)
    assert np.allclose(r, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_discretisation_error_closed_form():
    """e_disc of the main mode: DST solve against the closed form."""
    for n in (8, 16, 32):
        u = exact.mode(n, (1, 1, 1))
        uh = exact.dst_solve(3.0 * np.pi ** 2 * u)
        assert abs(np.abs(uh - u).max() - exact.e_disc_main(n)) < 1e-12
    e = [exact.e_disc_main(n) for n in (32, 64, 128, 256)]
    assert abs(e[0] - 8.0068e-4) < 1e-7
    for a, b in zip(e, e[1:]):
        assert 3.9 < a / b < 4.1
