"""A second, independent implementation of FMG and SR-FMG, used to cross-check
the oracle's box bookkeeping.

Every segment level is a whole padded level grid; the segment's regions of
Sec. 4 (compute region Omega^C, its ghost shell inside the domain Omega^GSR,
the support Omega^F, the genuine level-0 cells) are boolean masks.  Cells a
segment does not own start as NaN, so any read outside the regions the paper
allows shows up as NaN in the result.  Transfers are applied dimension by
dimension, the coarsest solve uses the DST (exact.dst_solve_g) instead of
elimination, and restriction uses reshape/mean: the arithmetic order differs
from the oracle's, the results agree to rounding.

Readings follow the oracle's (A = -Delta_h with the 7-point or a 27-point
stencil, ghost = -mirror, Chebyshev on D^-1 A over [lo, hi] * lambda_max,
averaging restriction, trilinear prolongation, owner-writes at the
transition level).  Grids cover [0, l0] x [0, l1] x [0, l2] with n cells per
unit length; arrays are [z][y][x].
"""
import itertools

import numpy as np

import exact


class Params:
    def __init__(self, alpha=1, nu1=2, nu2=2, cheb_lo=1.0 / 6.0, cheb_hi=1.0,
                 lengths=(1, 1, 1), stencil=7, weights=None):
        self.alpha, self.nu1, self.nu2 = alpha, nu1, nu2
        self.lo, self.hi = cheb_lo, cheb_hi
        self.lengths = tuple(int(v) for v in lengths)
        self.stencil = stencil
        self.w = (1.0, 0.0, 0.0) if stencil == 7 else tuple(weights)
        w1, w2, w3 = self.w
        self.w0 = 6 * w1 + 12 * w2 + 8 * w3
        # largest value of the multilinear symbol over [-1, 1]^3, at a corner
        self.lmax = max(exact.symbol(self.w, c) for c in itertools.product((-1, 1), repeat=3)) \
            / self.w0

    def shape(self, n):
        lx, ly, lz = self.lengths
        return (n * lz, n * ly, n * lx)


def pad(a, fill=0.0):
    p = np.full(tuple(s + 2 for s in a.shape), fill)
    p[1:-1, 1:-1, 1:-1] = a
    return p


def inner(p):
    return p[1:-1, 1:-1, 1:-1]


def fill_bc(p):
    """ghost = -mirror on the six domain faces, x then y then z."""
    p[:, :, 0] = -p[:, :, 1]
    p[:, :, -1] = -p[:, :, -2]
    p[:, 0, :] = -p[:, 1, :]
    p[:, -1, :] = -p[:, -2, :]
    p[0] = -p[1]
    p[-1] = -p[-2]


def _shifted(p, dz, dy, dx):
    nz, ny, nx = (s - 2 for s in p.shape)
    return p[1 + dz:1 + dz + nz, 1 + dy:1 + dy + ny, 1 + dx:1 + dx + nx]


def apply(p, n, P):
    """A u on the interior of the padded p (ghosts must be valid); h = 1/n."""
    sums = [0.0, 0.0, 0.0, 0.0]
    for dz, dy, dx in itertools.product((-1, 0, 1), repeat=3):
        far = (dz != 0) + (dy != 0) + (dx != 0)
        if far and P.w[far - 1] != 0.0:
            sums[far] = sums[far] + _shifted(p, dz, dy, dx)
    w1, w2, w3 = P.w
    return (P.w0 * inner(p) - w1 * sums[1] - w2 * sums[2] - w3 * sums[3]) * float(n * n)


def restrict(a):
    z, y, x = (s // 2 for s in a.shape)
    return a.reshape(z, 2, y, 2, x, 2).mean(axis=(1, 3, 5))


def _prolong1d(p, axis):
    p = np.moveaxis(p, axis, 0)
    nc = p.shape[0] - 2
    c, lft, rgt = p[1:-1], p[:-2], p[2:]
    out = np.empty((2 * nc,) + p.shape[1:])
    out[0::2] = 0.75 * c + 0.25 * lft
    out[1::2] = 0.75 * c + 0.25 * rgt
    return np.moveaxis(out, 0, axis)


def prolong(p):
    """trilinear interpolation of a padded coarse grid onto the fine interior
    (x, then y, then z; each pass drops the padding of its own axis)."""
    return _prolong1d(_prolong1d(_prolong1d(p, 2), 1), 0)


def cheb(p, f, mask, n, nu, P):
    """Chebyshev smoother on the cells of mask; p is updated in place."""
    if nu <= 0:
        return
    a, b = P.lo * P.lmax, P.hi * P.lmax
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    dinv = 1.0 / (P.w0 * n * n)
    fill_bc(p)
    d = dinv * (f - apply(p, n, P)) / theta
    rho_old = delta / theta
    for m in range(nu):
        u = inner(p)
        u[mask] += d[mask]
        if m == nu - 1:
            break
        fill_bc(p)
        r = dinv * (f - apply(p, n, P))
        rho = 1.0 / (2.0 * theta / delta - rho_old)
        d = rho * rho_old * d + (2.0 * rho / delta) * r
        rho_old = rho


def _direct(f, n, P):
    return exact.dst_solve_g(f, n, P.w)


def fasmgv(p, rhs, n, P, coarsest):
    """FAS V-cycle on a whole padded grid p (updated in place), n per unit."""
    if n <= coarsest:
        inner(p)[...] = _direct(rhs, n, P)
        return
    full = np.ones(rhs.shape, dtype=bool)
    cheb(p, rhs, full, n, P.nu1, P)
    fill_bc(p)
    r = rhs - apply(p, n, P)
    pc = pad(restrict(inner(p)))
    fill_bc(pc)
    t = pc.copy()
    rc = restrict(r) + apply(pc, n // 2, P)
    fasmgv(pc, rc, n // 2, P, coarsest)
    e = pc - t
    fill_bc(e)
    inner(p)[...] += prolong(e)
    cheb(p, rhs, full, n, P.nu2, P)


def _coarsest(n):
    while n > 3:
        n //= 2
    return n


def fmg(f, P, coarsest=None, n=None):
    """Full multigrid on the whole grid; returns the padded finest solution."""
    n = f.shape[2] // P.lengths[0] if n is None else n
    coarsest = _coarsest(n) if coarsest is None else coarsest
    fs, ns = [f], [n]
    while ns[-1] > coarsest:
        fs.append(restrict(fs[-1]))
        ns.append(ns[-1] // 2)
    fs, ns = fs[::-1], ns[::-1]
    p = pad(_direct(fs[0], ns[0], P))
    for fk, nk in zip(fs[1:], ns[1:]):
        fill_bc(p)
        q = pad(prolong(p))
        cheb(q, fk, np.ones(fk.shape, dtype=bool), nk, P.alpha, P)
        fasmgv(q, fk, nk, P, coarsest)
        p = q
    return p


def box_mask(shape, lo, hi):
    m = np.zeros(shape, dtype=bool)
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


def sr_fmg(f, seg, K, J, P, coarsest=None):
    """FASFMGSR with full-grid masks; returns u on the fine grid.  coarsest:
    cells per unit length of the exactly solved grid (default: halve to 2
    or 3)."""
    n = f.shape[2] // P.lengths[0]
    nk = [n >> (K - k) for k in range(K + 1)]
    dims = lambda k: [nk[k] * l for l in P.lengths]  # noqa: E731  (x, y, z)
    fsr = {K: f}
    for k in range(K, 0, -1):
        fsr[k - 1] = restrict(fsr[k])
    coarsest = _coarsest(nk[0]) if coarsest is None else coarsest
    u0 = fmg(fsr[0], P, coarsest, nk[0])
    rho0 = np.full(P.shape(nk[0]), np.nan)
    uhat0 = np.full(P.shape(nk[0]), np.nan)
    nsd = [n * l // seg for l in P.lengths]
    segs = []
    for pz in range(nsd[2]):
        for py in range(nsd[1]):
            for px in range(nsd[0]):
                q = (px, py, pz)
                s = {"C": {}, "CG": {}, "F": {}, "U": {}, "T": {}, "R": {}}
                for k in range(1, K + 1):
                    sk = seg >> (K - k)
                    nd = dims(k)
                    lo = [max(0, qd * sk - J[k - 1]) for qd in q]
                    hi = [min(nd[d], (q[d] + 1) * sk + J[k - 1]) for d in range(3)]
                    sh = P.shape(nk[k])
                    s["C"][k] = box_mask(sh, lo, hi)
                    s["CG"][k] = box_mask(sh, [max(0, v - 1) for v in lo],
                                          [min(nd[d], hi[d] + 1) for d in range(3)])
                    s["F"][k - 1] = box_mask(P.shape(nk[k - 1]), [v // 2 for v in lo],
                                             [v // 2 for v in hi])
                    s["U"][k] = np.full(tuple(v + 2 for v in sh), np.nan)
                    s["T"][k] = np.full(tuple(v + 2 for v in sh), np.nan)
                    s["R"][k] = np.full(sh, np.nan)
                s0 = seg >> K
                s["G0"] = box_mask(P.shape(nk[0]), [qd * s0 for qd in q],
                                   [(qd + 1) * s0 for qd in q])
                s["GK"] = box_mask(P.shape(n), [qd * seg for qd in q],
                                   [(qd + 1) * seg for qd in q])
                segs.append(s)
    for k in range(1, K + 1):
        fill_bc(u0)
        for s in segs:
            if k == 1:
                src = u0
            else:
                src = s["U"][k - 1]
                fill_bc(src)
            pr = prolong(src)
            inner(s["U"][k])[s["CG"][k]] = pr[s["CG"][k]]
            s["R"][k][s["C"][k]] = fsr[k][s["C"][k]]
            cheb(s["U"][k], s["R"][k], s["C"][k], nk[k], P.alpha, P)
            for j in range(k, 0, -1):
                U = s["U"][j]
                cheb(U, s["R"][j], s["C"][j], nk[j], P.nu1, P)
                fill_bc(U)
                r = s["R"][j] - apply(U, nk[j], P)
                uc, rc = restrict(inner(U)), restrict(r)
                if j > 1:
                    F = s["F"][j - 1]
                    Uc = s["U"][j - 1]
                    inner(Uc)[F] = uc[F]
                    fill_bc(Uc)
                    s["T"][j - 1] = Uc.copy()
                    Au = apply(Uc, nk[j - 1], P)
                    C = s["C"][j - 1]
                    s["R"][j - 1][C] = Au[C]
                    s["R"][j - 1][F] += rc[F]
                else:
                    g = s["G0"]
                    uhat0[g] = uc[g]
                    rho0[g] = rc[g]
        inner(u0)[...] = uhat0
        fill_bc(u0)
        t0 = u0.copy()
        rhs0 = rho0 + apply(u0, nk[0], P)
        fasmgv(u0, rhs0, nk[0], P, coarsest)
        e0 = u0 - t0
        fill_bc(e0)
        for s in segs:
            for j in range(1, k + 1):
                if j == 1:
                    e = e0
                else:
                    e = s["U"][j - 1] - s["T"][j - 1]
                    fill_bc(e)
                pr = prolong(e)
                CG = s["CG"][j]
                inner(s["U"][j])[CG] += pr[CG]
                cheb(s["U"][j], s["R"][j], s["C"][j], nk[j], P.nu2, P)
    u = np.full(P.shape(n), np.nan)
    for s in segs:
        u[s["GK"]] = inner(s["U"][K])[s["GK"]]
    return u
