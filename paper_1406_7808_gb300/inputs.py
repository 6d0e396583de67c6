"""Seeded synthetic inputs for the 3D Poisson problem on the unit cube.

This module holds the problem set-up only (manufactured solutions and the
right-hand sides they imply); it contains none of the solver's arithmetic and
imports nothing from the solver or from the CPU oracle, so both can be fed
the same arrays.

Grid: N^3 cells of the unit cube, cell centres x_i = (i + 1/2)/N (Sec. 2,
Eq. eq:deq); arrays are float64 with index order [z][y][x].

Manufactured solution (the workload of every configuration):
    u(x) = sin(pi x) sin(pi y) sin(pi z)
           + sum_{m=1..8} a_m sin(k_{m,x} pi x) sin(k_{m,y} pi y) sin(k_{m,z} pi z)
with a_m ~ N(0, sigma = 1e-3) and integer wavenumbers k uniform in [1, 4],
drawn from ``numpy.random.default_rng(seed)`` in the order a, then k.
It vanishes on the boundary, and f = -Delta u is evaluated analytically at the
cell centres.
"""
import numpy as np

MODES = 8
SIGMA = 1e-3
KMAX = 4


def cell_centres(n):
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def _draw(seed, modes=MODES, sigma=SIGMA, kmax=KMAX):
    rng = np.random.default_rng(seed)
    a = rng.normal(0.0, sigma, size=modes)
    k = rng.integers(1, kmax + 1, size=(modes, 3))
    return a, k


def _product(n, kx, ky, kz):
    x = cell_centres(n)
    sx = np.sin(kx * np.pi * x)
    sy = np.sin(ky * np.pi * x)
    sz = np.sin(kz * np.pi * x)
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def manufactured(n, seed, *, sigma=SIGMA, modes=MODES, main=True):
    """Return (f, u_exact) on the n^3 cell centres; f = -Delta u_exact."""
    a, k = _draw(seed, modes, sigma)
    u = np.zeros((n, n, n))
    f = np.zeros((n, n, n))
    if main:
        m = _product(n, 1, 1, 1)
        u += m
        f += 3.0 * np.pi ** 2 * m
    for am, (kx, ky, kz) in zip(a, k):
        m = _product(n, int(kx), int(ky), int(kz))
        u += am * m
        f += am * np.pi ** 2 * float(kx * kx + ky * ky + kz * kz) * m
    return f, u


def smooth_noise(n, seed, *, sigma=SIGMA, modes=MODES):
    """A seeded sum of low sine modes (amplitudes N(0, sigma)); zero on the boundary."""
    _, u = manufactured(n, seed, sigma=sigma, modes=modes, main=False)
    return u


def target(n, seed_u=0, seed_noise=2):
    """u_target = manufactured u (seed_u) + smooth noise (seed_noise), for the loss
    0.5 ||u(f) - u_target||^2 of the differentiable solve."""
    _, u = manufactured(n, seed_u)
    return u + smooth_noise(n, seed_noise)


def random_direction(n, rng):
    """A random smooth direction in f-space (for finite-difference checks)."""
    seed = int(rng.integers(0, 2 ** 31 - 1))
    f, _ = manufactured(n, seed, sigma=1.0, main=False)
    return f
