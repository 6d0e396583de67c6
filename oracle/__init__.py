"""CPU oracle for FAS-FMG and segmental-refinement FAS-FMG (FP64, plain C).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may load this package; the product path never
does.  The C source (``srfmg_oracle.c``) shares no code with the CUDA library.

Arrays are numpy float64, shape (n, n, n), index order [z][y][x] (x fastest).
Every function returns new arrays and leaves its inputs untouched.

Paper: Adams, Brown, Knepley, Samtaney, "Segmental Refinement: A Multigrid
Technique for Data Locality" -- Sec. 3 (FASMGV, FMG), Sec. 4 (FASFMGSR,
FASMGVSR, Eq. eq:nb), Sec. 5.1 (components).
"""
import ctypes
import os

import numpy as np

from . import build as _build

MAXK = 12


class OrConfig(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int),
        ("seg", ctypes.c_int),
        ("K", ctypes.c_int),
        ("J", ctypes.c_int * MAXK),
        ("alpha", ctypes.c_int),
        ("nu1", ctypes.c_int),
        ("nu2", ctypes.c_int),
        ("cheb_lo", ctypes.c_double),
        ("cheb_hi", ctypes.c_double),
        ("reverse_segments", ctypes.c_int),
        ("n_threads", ctypes.c_int),
        ("n_coarse", ctypes.c_int),
        ("len", ctypes.c_int * 3),
        ("stencil", ctypes.c_int),
        ("w", ctypes.c_double * 3),
    ]


_LIB = None
_DP = ctypes.POINTER(ctypes.c_double)


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        for name in ("or_solve", "or_vcycle"):
            getattr(lib, name).argtypes = [ctypes.POINTER(OrConfig), _DP, _DP]
            getattr(lib, name).restype = ctypes.c_int
        lib.or_vsolve.argtypes = [ctypes.POINTER(OrConfig), _DP, _DP, ctypes.c_double,
                                  ctypes.c_int, ctypes.POINTER(ctypes.c_int), _DP]
        lib.or_vsolve.restype = ctypes.c_int
        lib.or_check_config.argtypes = [ctypes.POINTER(OrConfig)]
        PC = ctypes.POINTER(OrConfig)
        for name in ("or_apply_g", "or_restrict_g", "or_prolong_g", "or_coarse_solve_g"):
            getattr(lib, name).argtypes = [PC, _DP, _DP]
        lib.or_smooth_g.argtypes = [PC, ctypes.c_int, _DP, _DP]
        lib.or_residual_g.argtypes = [PC, _DP, _DP, _DP]
        lib.or_buffer_schedule.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_int)]
        lib.or_buffer_schedule.restype = None
        lib.or_max_threads.restype = ctypes.c_int
        _LIB = lib
    return _LIB


def _p(a):
    return a.ctypes.data_as(_DP)


def _grid(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 3:
        raise ValueError("expected a 3D array")
    if shape is not None and a.shape != tuple(shape):
        raise ValueError("grid size mismatch")
    return a


def per_unit(a, lengths=(1, 1, 1)):
    """Cells per unit length n of an array of shape (n len2, n len1, n len0)
    ([z][y][x]) on the domain [0, len0] x [0, len1] x [0, len2]."""
    lx, ly, lz = (int(v) for v in lengths)
    nz, ny, nx = a.shape
    n = nx // lx
    if n < 1 or (nz, ny, nx) != (n * lz, n * ly, n * lx):
        raise ValueError(f"shape {a.shape} does not match the domain lengths {lengths}")
    return n


def _check(st, what):
    if st != 0:
        raise RuntimeError(f"oracle {what} failed with status {st}")


def buffer_schedule(A, B, K):
    """J_k = 2 floor((A + B (K - k)) / 2) for k = 1..K (Eq. eq:nb)."""
    J = (ctypes.c_int * max(K, 1))()
    _lib().or_buffer_schedule(A, B, K, J)
    return [J[i] for i in range(K)]


def mbs_schedule(J1, K):
    """Maximum buffer schedule (Sec. 5.2.1): the coarser compute regions are
    exactly the supports of the finer ones, Omega^C_k = Omega^F_k for k < K,
    i.e. J_{k+1} = 2 J_k, starting from J_1."""
    J = [J1]
    for _ in range(K - 1):
        J.append(2 * J[-1])
    return J


def make_config(n, seg=0, K=0, J=None, A=4, B=1, alpha=1, nu1=2, nu2=2,
                cheb_lo=1.0 / 6.0, cheb_hi=1.0, reverse_segments=False, n_threads=0,
                n_coarse=0, lengths=(1, 1, 1), stencil=7, weights=None):
    """n: cells per unit length; lengths: the domain [0, l0] x [0, l1] x [0, l2];
    stencil 7 or 27 with weights (faces, edges, corners) of the 27-point operator."""
    c = OrConfig()
    c.n, c.seg, c.K = n, seg, K
    if K > 0:
        Js = list(J) if J is not None else buffer_schedule(A, B, K)
        if len(Js) != K:
            raise ValueError("J must have K entries")
        for i, v in enumerate(Js):
            c.J[i] = int(v)
    c.alpha, c.nu1, c.nu2 = alpha, nu1, nu2
    c.cheb_lo, c.cheb_hi = cheb_lo, cheb_hi
    c.reverse_segments = int(bool(reverse_segments))
    c.n_threads = n_threads
    c.n_coarse = n_coarse
    for d in range(3):
        c.len[d] = int(lengths[d])
    c.stencil = int(stencil)
    if weights is None and int(stencil) == 27:
        weights = W27_DEFAULT
    if weights is not None:
        for d in range(3):
            c.w[d] = float(weights[d])
    return c


# the 27-point reading used when no weights are given: (14, 3, 1)/30 for the
# face, edge and corner neighbours (centre 128/30)
W27_DEFAULT = (14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)


GEO_KEYS = ("lengths", "stencil", "weights")


def _geo(kw):
    return {k: kw[k] for k in GEO_KEYS if k in kw}


def _cfg_for(a, kw):
    """configuration for array a (its n from the domain lengths in kw)"""
    return make_config(per_unit(a, kw.get("lengths", (1, 1, 1))), **kw)


def check_config(**kw):
    """0 if the oracle accepts the configuration, a negative code otherwise."""
    return _lib().or_check_config(ctypes.byref(make_config(**kw)))


def solve(f, **kw):
    """FMG (seg=0 or K=0) or SR-FMG (FASFMGSR) of A u = f; returns u."""
    f = _grid(f)
    c = _cfg_for(f, kw)
    u = np.zeros_like(f)
    _check(_lib().or_solve(ctypes.byref(c), _p(f), _p(u)), "solve")
    return u


def solve_refined(f, n_outer=2, **kw):
    """Defect correction around FMG / SR-FMG, all in float64:
    u = S(f), then n_outer - 1 times u += S(f - A u).  The mixed-precision
    mode runs the same loop with S in float32; this is its float64 reference."""
    f = _grid(f)
    u = solve(f, **kw)
    for _ in range(n_outer - 1):
        u = u + solve(residual(u, f, **_geo(kw)), **kw)
    return u


def _plain_kw(kw):
    return {k: v for k, v in kw.items() if k not in ("seg", "K", "J", "A", "B")}


def vcycle(f, u, **kw):
    """One FAS V-cycle FASMGV(L, u, f) on the global grid; returns the new u."""
    f = _grid(f)
    u = _grid(u, f.shape).copy()
    c = _cfg_for(f, _plain_kw(kw))
    _check(_lib().or_vcycle(ctypes.byref(c), _p(f), _p(u)), "vcycle")
    return u


def vsolve(f, u0=None, rtol=1e-4, max_cycles=100, **kw):
    """Iterative V-cycle solver (the comparison solver of Sec. 5.3): FASMGV
    from u0 (zero by default) until ||f - A u||_inf <= rtol ||f||_inf.
    Returns (u, cycles, relative residual)."""
    f = _grid(f)
    u = np.zeros_like(f) if u0 is None else _grid(u0, f.shape).copy()
    c = _cfg_for(f, _plain_kw(kw))
    cycles = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    _check(_lib().or_vsolve(ctypes.byref(c), _p(f), _p(u), float(rtol), int(max_cycles),
                            ctypes.byref(cycles), ctypes.byref(rel)), "vsolve")
    return u, cycles.value, rel.value


def apply(u, **geo):
    """A u (7-point A = -Delta_h by default; Dirichlet ghosts, Sec. 3.3)."""
    u = _grid(u)
    out = np.empty_like(u)
    _check(_lib().or_apply_g(ctypes.byref(_cfg_for(u, geo)), _p(u), _p(out)), "apply")
    return out


def residual(u, f, **geo):
    u = _grid(u)
    f = _grid(f, u.shape)
    r = np.empty_like(u)
    _check(_lib().or_residual_g(ctypes.byref(_cfg_for(u, geo)), _p(f), _p(u), _p(r)),
           "residual")
    return r


def smooth(u, f, nu, cheb_lo=1.0 / 6.0, cheb_hi=1.0, **geo):
    """Chebyshev smoother S^nu(L, u, f) on the whole grid; returns the new u."""
    u = _grid(u).copy()
    f = _grid(f, u.shape)
    c = _cfg_for(u, dict(geo, cheb_lo=cheb_lo, cheb_hi=cheb_hi))
    _check(_lib().or_smooth_g(ctypes.byref(c), nu, _p(f), _p(u)), "smooth")
    return u


def restrict(a, **geo):
    """8-child average onto the grid with half the cells per dimension."""
    a = _grid(a)
    out = np.empty(tuple(s // 2 for s in a.shape))
    _check(_lib().or_restrict_g(ctypes.byref(_cfg_for(a, geo)), _p(a), _p(out)), "restrict")
    return out


def prolong(ac, **geo):
    """Cell-centred trilinear interpolation onto the grid with twice the cells
    per dimension."""
    ac = _grid(ac)
    out = np.empty(tuple(2 * s for s in ac.shape))
    _check(_lib().or_prolong_g(ctypes.byref(_cfg_for(ac, geo)), _p(ac), _p(out)), "prolong")
    return out


def coarse_solve(f, **geo):
    """Exact solve of A u = f by a banded Cholesky factorisation (small grids)."""
    f = _grid(f)
    u = np.empty_like(f)
    _check(_lib().or_coarse_solve_g(ctypes.byref(_cfg_for(f, geo)), _p(f), _p(u)),
           "coarse_solve")
    return u


def max_threads():
    return _lib().or_max_threads()


LIBRARY = _build.LIBRARY
