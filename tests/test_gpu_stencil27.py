"""GPU parity on the paper's own model problem (Sec. 5.1): rectangular
domains and the 27-point operator, through the C ABI, against the oracle
(FP64, 1e-11 relative max-norm): every component on rectangles and both
27-point readings, plain FMG, SR-FMG on 4 x 2 x 2 segment layouts, the
V-cycle solver, the mixed-precision mode on a rectangle (7-point), and one
configuration of Table 1 (256 x 128 x 128 cells, K = 4, N0V = 4) cell by
cell."""
import numpy as np
import pytest

from paper_1406_7808_gb300 import inputs

pytestmark = pytest.mark.gpu
TOL = 1e-11
SIMPSON = (0.0, 1.0 / 6.0, 1.0 / 12.0)
W1430 = (14.0 / 30.0, 3.0 / 30.0, 1.0 / 30.0)
RECT = (2, 1, 1)
OPS = [dict(lengths=RECT), dict(lengths=RECT, stencil=27, weights=SIMPSON),
       dict(lengths=RECT, stencil=27, weights=W1430),
       dict(lengths=(1, 3, 2), stencil=27, weights=W1430)]


def T(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def shape_of(n, lengths):
    return (n * lengths[2], n * lengths[1], n * lengths[0])


@pytest.mark.parametrize("geo", OPS)
def test_components(gpu, oracle_mod, geo):
    rng = np.random.default_rng(3)
    n = 8
    sh = shape_of(n, geo["lengths"])
    u, f = rng.standard_normal(sh), rng.standard_normal(sh)
    assert rel(gpu.op_apply(T(u), **geo).cpu().numpy(), oracle_mod.apply(u, **geo)) < TOL
    assert rel(gpu.op_residual(T(u), T(f), **geo).cpu().numpy(),
               oracle_mod.residual(u, f, **geo)) < TOL
    for nu in (1, 2, 3):
        assert rel(gpu.op_smooth(T(u), T(f), nu, **geo).cpu().numpy(),
                   oracle_mod.smooth(u, f, nu, **geo)) < TOL
    assert rel(gpu.op_restrict(T(u), **geo).cpu().numpy(), oracle_mod.restrict(u, **geo)) < TOL
    assert rel(gpu.op_prolong(T(u), **geo).cpu().numpy(), oracle_mod.prolong(u, **geo)) < TOL
    fc = rng.standard_normal(shape_of(2, geo["lengths"]))
    assert rel(gpu.op_coarse_solve(T(fc), **geo).cpu().numpy(),
               oracle_mod.coarse_solve(fc, **geo)) < TOL


def gpu_solve(gpu, f, n, **kw):
    with gpu.Solver(n, **kw) as s:
        return s.solve(T(f)).cpu().numpy()


@pytest.mark.parametrize("geo", OPS[:3])
@pytest.mark.parametrize("n", [2, 4, 8, 16, 32])
def test_plain_fmg(gpu, oracle_mod, geo, n):
    f, _ = inputs.paper_problem(n, lengths=geo["lengths"], R=geo["lengths"])
    assert rel(gpu_solve(gpu, f, n, **geo), oracle_mod.solve(f, **geo)) < TOL


SR = [(8, dict(seg=4, K=1, J=[2])), (16, dict(seg=8, K=2, J=[2, 4])),
      (16, dict(seg=8, K=2, J=[4, 4])), (16, dict(seg=4, K=2, J=[2, 2])),
      (32, dict(seg=16, K=3, J=[4, 4, 4])), (32, dict(seg=16, K=2, A=4, B=1)),
      (32, dict(seg=16, K=3, A=4, mbs=True))]


def _oracle_kw(kw):
    kw = dict(kw)
    if kw.pop("mbs", False):
        J1 = kw.pop("A")
        kw["J"] = [J1 << k for k in range(kw["K"])]
    elif "J" not in kw:
        from oracle import buffer_schedule
        kw["J"] = buffer_schedule(kw.pop("A"), kw.pop("B"), kw["K"])
    return kw


@pytest.mark.parametrize("geo", OPS[:3])
@pytest.mark.parametrize("n,kw", SR)
def test_sr_fmg(gpu, oracle_mod, geo, n, kw):
    f, _ = inputs.paper_problem(n)
    ref = oracle_mod.solve(f, **_oracle_kw(kw), **geo)
    assert rel(gpu_solve(gpu, f, n, **kw, **geo), ref) < TOL


@pytest.mark.parametrize("geo", OPS[1:3])
def test_vsolve(gpu, oracle_mod, geo):
    n = 16
    f, _ = inputs.paper_problem(n)
    ur, cr, qr = oracle_mod.vsolve(f, rtol=1e-6, **geo)
    with gpu.Solver(n, **geo) as s:
        u, c, q = s.vsolve(T(f), rtol=1e-6)
    assert c == cr
    assert rel(u.cpu().numpy(), ur) < TOL


def test_mixed_precision_rectangle(gpu, oracle_mod):
    """float32 SR-FMG inside float64 defect correction on [0,2]x[0,1]^2
    (7-point): within 0.1 e_disc of the float64 loop."""
    n = 64
    f, uex = inputs.paper_problem(n)
    kw = dict(seg=32, K=2, J=[8, 8], lengths=RECT)
    ref = oracle_mod.solve_refined(f, 2, **kw)
    u = gpu_solve(gpu, f, n, mixed=True, n_outer=2, **kw)
    e_disc = np.abs(oracle_mod.vsolve(f, rtol=1e-13, max_cycles=60, lengths=RECT)[0] - uex).max()
    assert np.abs(u - ref).max() <= 0.1 * e_disc


def test_table1_configuration(gpu, oracle_mod):
    """Table 1, column log2 N0V = 2 (K = 4), A = 8, B = 0: 64^3-cell segments
    on the 256 x 128 x 128 grid, 27-point operator; every cell against the
    oracle, and the error ratio e_r = e_SR / e_conv the same on both."""
    n = 128
    geo = dict(lengths=RECT, stencil=27, weights=W1430)
    kw = dict(seg=64, K=4, A=8, B=0)
    f, uex = inputs.paper_problem(n)
    ref = oracle_mod.solve(f, **_oracle_kw(kw), **geo)
    u = gpu_solve(gpu, f, n, **kw, **geo)
    assert rel(u, ref) < TOL
    plain = gpu_solve(gpu, f, n, **geo)
    e_r = np.abs(u - uex).max() / np.abs(plain - uex).max()
    e_r_ref = np.abs(ref - uex).max() / np.abs(oracle_mod.solve(f, **geo) - uex).max()
    assert e_r == pytest.approx(e_r_ref, rel=1e-8)
