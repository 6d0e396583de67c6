"""A second, independent implementation of FMG and SR-FMG, used to cross-check
the oracle's box bookkeeping.

Every segment level is a whole padded level grid; the segment's regions of
Sec. 4 (compute region Omega^C, its ghost shell inside the domain Omega^GSR,
the support Omega^F, the genuine level-0 cells) are boolean masks.  Cells a
segment does not own start as NaN, so any read outside the regions the paper
allows shows up as NaN in the result.  Transfers are applied dimension by
dimension, the coarsest solve uses the DST (exact.dst_solve) instead of
elimination, and restriction uses reshape/mean: the arithmetic order differs
from the oracle's, the results agree to rounding.

Readings follow the oracle's (A = -Delta_h, ghost = -mirror, Chebyshev on
D^-1 A over [lo, hi] * 2, averaging restriction, trilinear prolongation,
owner-writes at the transition level).
"""
import numpy as np

from exact import dst_solve


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


def apply(p, n):
    c = p[1:-1, 1:-1, 1:-1]
    nb = (p[:-2, 1:-1, 1:-1] + p[2:, 1:-1, 1:-1] + p[1:-1, :-2, 1:-1]
          + p[1:-1, 2:, 1:-1] + p[1:-1, 1:-1, :-2] + p[1:-1, 1:-1, 2:])
    return (6.0 * c - nb) * float(n * n)


def restrict(a):
    m = a.shape[0] // 2
    return a.reshape(m, 2, m, 2, m, 2).mean(axis=(1, 3, 5))


def _prolong1d(p, axis):
    p = np.moveaxis(p, axis, 0)
    nc = p.shape[0] - 2
    c, lft, rgt = p[1:-1], p[:-2], p[2:]
    out = np.empty((2 * nc,) + p.shape[1:])
    out[0::2] = 0.75 * c + 0.25 * lft
    out[1::2] = 0.75 * c + 0.25 * rgt
    return np.moveaxis(out, 0, axis)


def prolong(p):
    """trilinear interpolation of a padded coarse grid onto the fine interior."""
    return _prolong1d(_prolong1d(_prolong1d(p, 2), 1), 0)


def cheb(p, f, mask, n, nu, lo, hi):
    """Chebyshev smoother on the cells of mask; p is updated in place."""
    if nu <= 0:
        return
    a, b = 2.0 * lo, 2.0 * hi
    theta, delta = 0.5 * (a + b), 0.5 * (b - a)
    dinv = 1.0 / (6.0 * n * n)
    fill_bc(p)
    d = dinv * (f - apply(p, n)) / theta
    rho_old = delta / theta
    for m in range(nu):
        u = inner(p)
        u[mask] += d[mask]
        if m == nu - 1:
            break
        fill_bc(p)
        r = dinv * (f - apply(p, n))
        rho = 1.0 / (2.0 * theta / delta - rho_old)
        d = rho * rho_old * d + (2.0 * rho / delta) * r
        rho_old = rho


class Params:
    def __init__(self, alpha=1, nu1=2, nu2=2, cheb_lo=1.0 / 6.0, cheb_hi=1.0):
        self.alpha, self.nu1, self.nu2 = alpha, nu1, nu2
        self.lo, self.hi = cheb_lo, cheb_hi


def fasmgv(p, rhs, P, coarsest):
    """FAS V-cycle on a whole padded grid p (updated in place)."""
    n = p.shape[0] - 2
    if n <= coarsest:
        inner(p)[...] = dst_solve(rhs)
        return
    full = np.ones((n,) * 3, dtype=bool)
    cheb(p, rhs, full, n, P.nu1, P.lo, P.hi)
    fill_bc(p)
    r = rhs - apply(p, n)
    pc = pad(restrict(inner(p)))
    fill_bc(pc)
    t = pc.copy()
    rc = restrict(r) + apply(pc, n // 2)
    fasmgv(pc, rc, P, coarsest)
    e = pc - t
    fill_bc(e)
    inner(p)[...] += prolong(e)
    cheb(p, rhs, full, n, P.nu2, P.lo, P.hi)


def _coarsest(n):
    while n > 3:
        n //= 2
    return n


def fmg(f, P, coarsest=None):
    """Full multigrid on the whole grid; returns the padded finest solution."""
    n = f.shape[0]
    coarsest = _coarsest(n) if coarsest is None else coarsest
    fs = [f]
    while fs[-1].shape[0] > coarsest:
        fs.append(restrict(fs[-1]))
    fs = fs[::-1]
    p = pad(dst_solve(fs[0]))
    for fk in fs[1:]:
        fill_bc(p)
        q = pad(prolong(p))
        nk = fk.shape[0]
        cheb(q, fk, np.ones((nk,) * 3, dtype=bool), nk, P.alpha, P.lo, P.hi)
        fasmgv(q, fk, P, coarsest)
        p = q
    return p


def box_mask(n, lo, hi):
    m = np.zeros((n,) * 3, dtype=bool)
    m[lo[2]:hi[2], lo[1]:hi[1], lo[0]:hi[0]] = True
    return m


def sr_fmg(f, seg, K, J, P):
    """FASFMGSR with full-grid masks; returns u on the fine grid."""
    n = f.shape[0]
    nk = [n >> (K - k) for k in range(K + 1)]
    fsr = {K: f}
    for k in range(K, 0, -1):
        fsr[k - 1] = restrict(fsr[k])
    coarsest = _coarsest(nk[0])
    u0 = fmg(fsr[0], P, coarsest)
    rho0 = np.full((nk[0],) * 3, np.nan)
    uhat0 = np.full((nk[0],) * 3, np.nan)
    nseg1 = n // seg
    segs = []
    for pz in range(nseg1):
        for py in range(nseg1):
            for px in range(nseg1):
                q = (px, py, pz)
                s = {"C": {}, "CG": {}, "F": {}, "U": {}, "T": {}, "R": {}}
                for k in range(1, K + 1):
                    sk = seg >> (K - k)
                    lo = [max(0, qd * sk - J[k - 1]) for qd in q]
                    hi = [min(nk[k], (qd + 1) * sk + J[k - 1]) for qd in q]
                    s["C"][k] = box_mask(nk[k], lo, hi)
                    s["CG"][k] = box_mask(nk[k], [max(0, v - 1) for v in lo],
                                          [min(nk[k], v + 1) for v in hi])
                    s["F"][k - 1] = box_mask(nk[k - 1], [v // 2 for v in lo], [v // 2 for v in hi])
                    s["U"][k] = np.full((nk[k] + 2,) * 3, np.nan)
                    s["T"][k] = np.full((nk[k] + 2,) * 3, np.nan)
                    s["R"][k] = np.full((nk[k],) * 3, np.nan)
                s0 = seg >> K
                s["G0"] = box_mask(nk[0], [qd * s0 for qd in q], [(qd + 1) * s0 for qd in q])
                s["GK"] = box_mask(n, [qd * seg for qd in q], [(qd + 1) * seg for qd in q])
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
            cheb(s["U"][k], s["R"][k], s["C"][k], nk[k], P.alpha, P.lo, P.hi)
            for j in range(k, 0, -1):
                U = s["U"][j]
                cheb(U, s["R"][j], s["C"][j], nk[j], P.nu1, P.lo, P.hi)
                fill_bc(U)
                r = s["R"][j] - apply(U, nk[j])
                uc, rc = restrict(inner(U)), restrict(r)
                if j > 1:
                    F = s["F"][j - 1]
                    Uc = s["U"][j - 1]
                    inner(Uc)[F] = uc[F]
                    fill_bc(Uc)
                    s["T"][j - 1] = Uc.copy()
                    Au = apply(Uc, nk[j - 1])
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
        rhs0 = rho0 + apply(u0, nk[0])
        fasmgv(u0, rhs0, P, coarsest)
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
                cheb(s["U"][j], s["R"][j], s["C"][j], nk[j], P.nu2, P.lo, P.hi)
    u = np.full((n,) * 3, np.nan)
    for s in segs:
        u[s["GK"]] = inner(s["U"][K])[s["GK"]]
    return u
