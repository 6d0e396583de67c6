"""Exact discrete solutions and closed forms used to pin the oracle.

Nothing here calls the oracle.  The operator A = -Delta_h with Dirichlet
ghosts (ghost = -interior) is diagonalised by the DST-II basis
sin(k pi (i + 1/2) / n), k = 1..n, with 1D eigenvalues 4 n^2 sin^2(k pi / 2n);
scipy's DST-II / DST-III pair therefore gives the exact discrete solve.
"""
import numpy as np
from scipy.fft import dstn, idstn


def lam1(n):
    k = np.arange(1, n + 1)
    return 4.0 * n * n * np.sin(k * np.pi / (2.0 * n)) ** 2


def eigenvalue(n, k):
    """Eigenvalue of A for the mode with wavenumbers k = (kx, ky, kz)."""
    return float(sum(4.0 * n * n * np.sin(kd * np.pi / (2.0 * n)) ** 2 for kd in k))


def mode(n, k):
    """Cell-centre samples of sin(kx pi x) sin(ky pi y) sin(kz pi z), [z][y][x]."""
    x = (np.arange(n) + 0.5) / n
    sx, sy, sz = (np.sin(kd * np.pi * x) for kd in k)
    return sz[:, None, None] * sy[None, :, None] * sx[None, None, :]


def dst_solve(f, workers=8):
    """u = A^-1 f exactly (up to rounding) through the DST-II eigenbasis."""
    n = f.shape[0]
    L1 = lam1(n)
    L = L1[:, None, None] + L1[None, :, None] + L1[None, None, :]
    return idstn(dstn(f, type=2, workers=workers) / L, type=2, workers=workers)


def dense_matrix(n):
    """A as a dense matrix, built as a Kronecker sum of 1D second differences
    (flattened index (z n + y) n + x); the end rows carry the ghost reflection."""
    T = 2.0 * np.eye(n) - np.eye(n, k=1) - np.eye(n, k=-1)
    T[0, 0] += 1.0
    T[-1, -1] += 1.0
    T *= n * n
    I = np.eye(n)
    return (np.kron(np.kron(I, I), T) + np.kron(np.kron(I, T), I)
            + np.kron(np.kron(T, I), I))


# ---- general grids: [0, l0] x [0, l1] x [0, l2], n cells per unit length,
# ---- arrays [z][y][x]; operator weights w = (faces, edges, corners):
# ---- A u = n^2 (w0 u - w1 sum_faces - w2 sum_edges - w3 sum_corners)

def symbol(w, c):
    """h^2 times the eigenvalue of A on the sine mode with cos(theta_d) = c_d."""
    w1, w2, w3 = w
    w0 = 6 * w1 + 12 * w2 + 8 * w3
    return (w0 - 2 * w1 * (c[0] + c[1] + c[2])
            - 4 * w2 * (c[0] * c[1] + c[0] * c[2] + c[1] * c[2]) - 8 * w3 * c[0] * c[1] * c[2])


def _cos(N):
    return np.cos(np.arange(1, N + 1) * np.pi / N)


def dst_solve_g(f, n, w):
    """u = A^-1 f through the DST-II eigenbasis for any grid shape and any
    reflection-symmetric 27-point weights (the 7-point operator is w = (1, 0, 0))."""
    nz, ny, nx = f.shape
    cz, cy, cx = _cos(nz)[:, None, None], _cos(ny)[None, :, None], _cos(nx)[None, None, :]
    lam = n * n * symbol(w, (cx, cy, cz))
    return idstn(dstn(f, type=2) / lam, type=2)


def mode_g(shape, k):
    """Samples of the discrete sine mode with wavenumbers k = (kx, ky, kz) on a
    grid of shape (nz, ny, nx)."""
    nz, ny, nx = shape
    s = [np.sin(kd * np.pi * (np.arange(N) + 0.5) / N) for kd, N in zip(k, (nx, ny, nz))]
    return s[2][:, None, None] * s[1][None, :, None] * s[0][None, None, :]


def eigenvalue_g(shape, n, w, k):
    nz, ny, nx = shape
    c = [np.cos(kd * np.pi / N) for kd, N in zip(k, (nx, ny, nz))]
    return float(n * n * symbol(w, c))


def _neighbour_sum_1d(N):
    """u_{i-1} + u_{i+1} with the ghost reflection u_{-1} = -u_0, u_N = -u_{N-1}."""
    S = np.eye(N, k=1) + np.eye(N, k=-1)
    S[0, 0] -= 1.0
    S[-1, -1] -= 1.0
    return S


def dense_matrix_g(shape, n, w):
    """A as a dense matrix from Kronecker products of 1D neighbour sums: face
    neighbours are sums in one dimension, edges products over two, corners
    over three (the reflection signs multiply)."""
    nz, ny, nx = shape
    Sx, Sy, Sz = _neighbour_sum_1d(nx), _neighbour_sum_1d(ny), _neighbour_sum_1d(nz)
    Ix, Iy, Iz = np.eye(nx), np.eye(ny), np.eye(nz)

    def k3(a, b, c):  # z, y, x factors, flattened index (z ny + y) nx + x
        return np.kron(np.kron(a, b), c)
    w1, w2, w3 = w
    w0 = 6 * w1 + 12 * w2 + 8 * w3
    faces = k3(Iz, Iy, Sx) + k3(Iz, Sy, Ix) + k3(Sz, Iy, Ix)
    edges = k3(Iz, Sy, Sx) + k3(Sz, Iy, Sx) + k3(Sz, Sy, Ix)
    corners = k3(Sz, Sy, Sx)
    m = nx * ny * nz
    return n * n * (w0 * np.eye(m) - w1 * faces - w2 * edges - w3 * corners)


def e_disc_main(n):
    """max |u_h - u| for u = sin(pi x) sin(pi y) sin(pi z), n even:
    u_h = u * pi^2 h^2 / (4 sin^2(pi h / 2)) and max |u| over cells is cos^3(pi / 2n)."""
    h = 1.0 / n
    ratio = np.pi ** 2 * h * h / (4.0 * np.sin(np.pi * h / 2.0) ** 2)
    return abs(ratio - 1.0) * np.cos(np.pi / (2.0 * n)) ** 3


def chebyshev_factor(lam, nu, lo, hi):
    """p_nu(lam) = T_nu((theta - lam)/delta) / T_nu(theta/delta) for the Chebyshev
    smoother on D^-1 A over [lo, hi] * 2; T_nu evaluated in closed form."""
    a, b = 2.0 * lo, 2.0 * hi
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)

    def T(x):
        x = float(x)
        if abs(x) <= 1.0:
            return np.cos(nu * np.arccos(x))
        s = 1.0 if x > 0 or nu % 2 == 0 else -1.0
        return s * np.cosh(nu * np.arccosh(abs(x)))

    return T((theta - lam) / delta) / T(theta / delta)
