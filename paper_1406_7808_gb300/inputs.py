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


# ---------------------------------------------------------------------------
# The model problem of the paper's experiments (Sec. 5.1): the domain
# [0, 2] x [0, 1] x [0, 1] with the prescribed solution
#     u(x) = prod_{i=1..3} (x_i^4 - R_i^2 x_i^2),   R = (2, 1, 1),
# which vanishes on the whole boundary (x_i = 0 or x_i = R_i).  With
# g_i(t) = t^4 - R_i^2 t^2 and g_i'' = 12 t^2 - 2 R_i^2, f = -Delta u =
# -sum_i g_i''(x_i) prod_{j != i} g_j(x_j), evaluated at the cell centres.
PAPER_LENGTHS = (2, 1, 1)
PAPER_R = (2.0, 1.0, 1.0)


def paper_problem(n, lengths=PAPER_LENGTHS, R=PAPER_R):
    """(f, u) on the grid with n cells per unit length over [0, l0] x [0, l1] x
    [0, l2], arrays of shape (n l2, n l1, n l0) indexed [z][y][x]."""
    xs = [cell_centres(n * int(l)) * int(l) for l in lengths]  # centres in [0, l]
    g = [t ** 4 - r * r * t ** 2 for t, r in zip(xs, R)]
    g2 = [12.0 * t ** 2 - 2.0 * r * r for t, r in zip(xs, R)]

    def outer(ax, ay, az):
        return az[:, None, None] * ay[None, :, None] * ax[None, None, :]
    u = outer(g[0], g[1], g[2])
    f = -(outer(g2[0], g[1], g[2]) + outer(g[0], g2[1], g[2]) + outer(g[0], g[1], g2[2]))
    return f, u
