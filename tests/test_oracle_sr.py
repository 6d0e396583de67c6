"""Pins for the oracle's segmental refinement (Sec. 4: regions, Eq. eq:nb,
Figs. "FMG segmental refinement" and "FAS V-cycle segmental refinement").

- special cases that must reduce to plain FMG: one segment, and buffers that
  cover the whole level (J_k >= N_k);
- equality with an independent full-grid/mask implementation
  (tests/sr_masked.py) on several geometries, including clipped boxes and a
  grid that coarsens to 3^3;
- invariants: segment order and thread count do not change a bit of the
  result; the solve is linear in f;
- accuracy: the SR error ratio e_r = e_SR / e_conv (Sec. 5.2) improves with
  larger buffers.  The paper's absolute e_r values (Tables 1-3) come from a
  27-point stencil on another domain and do not pin this problem.
"""
import numpy as np
import pytest

import exact
import sr_masked
from paper_1406_7808_gb300 import inputs, workloads


def test_buffer_schedule_eq_nb(oracle_mod):
    assert oracle_mod.buffer_schedule(4, 1, 3) == [6, 4, 4]
    assert oracle_mod.buffer_schedule(8, 0, 5) == [8] * 5
    assert oracle_mod.buffer_schedule(2, 3, 4) == [10, 8, 4, 2]
    assert oracle_mod.buffer_schedule(3, 0, 2) == [2, 2]


@pytest.mark.parametrize("n,K", [(16, 1), (32, 2), (32, 3)])
def test_one_segment_is_plain_fmg(oracle_mod, n, K):
    f, _ = inputs.manufactured(n, 0)
    plain = oracle_mod.solve(f)
    sr = oracle_mod.solve(f, seg=n, K=K, A=4, B=1)
    assert np.array_equal(sr, plain)


@pytest.mark.parametrize("n,seg,K", [(16, 8, 1), (32, 8, 2), (32, 16, 3)])
def test_whole_level_buffers_are_plain_fmg(oracle_mod, n, seg, K):
    f, _ = inputs.manufactured(n, 1)
    plain = oracle_mod.solve(f)
    J = [n >> (K - k) for k in range(1, K + 1)]  # J_k = N_k: every box is the whole level
    sr = oracle_mod.solve(f, seg=seg, K=K, J=J)
    assert np.array_equal(sr, plain)


GEOMETRIES = [
    (16, 8, 1, [2]),
    (32, 8, 2, [4, 4]),
    (32, 16, 2, [2, 4]),
    (32, 8, 3, [6, 4, 4]),
    (24, 12, 2, [2, 2]),
    (48, 16, 2, [4, 2]),
    (32, 8, 2, [0, 0]),
    (64, 16, 3, [2, 4, 8]),   # maximum buffer schedule (Sec. 5.2.1)
]


@pytest.mark.parametrize("n,seg,K,J", GEOMETRIES)
def test_matches_independent_masked_implementation(oracle_mod, n, seg, K, J):
    f, _ = inputs.manufactured(n, 1)
    a = oracle_mod.solve(f, seg=seg, K=K, J=J)
    b = sr_masked.sr_fmg(f, seg, K, J, sr_masked.Params())
    assert not np.isnan(b).any()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_masked_plain_fmg_matches(oracle_mod):
    for n in (8, 16, 24):
        f, _ = inputs.manufactured(n, 0)
        a = oracle_mod.solve(f)
        b = sr_masked.inner(sr_masked.fmg(f, sr_masked.Params()))
        assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_segment_order_and_threads_do_not_matter(oracle_mod):
    n = 64
    f, _ = inputs.manufactured(n, 2)
    kw = dict(seg=16, K=2, A=4, B=1)
    a = oracle_mod.solve(f, n_threads=1, **kw)
    b = oracle_mod.solve(f, n_threads=1, reverse_segments=True, **kw)
    c = oracle_mod.solve(f, n_threads=4, **kw)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


def test_sr_linear_in_f(oracle_mod):
    n = 32
    f1, _ = inputs.manufactured(n, 5)
    f2, _ = inputs.manufactured(n, 6)
    kw = dict(seg=8, K=2, A=4, B=1)
    lhs = oracle_mod.solve(2.0 * f1 - 0.5 * f2, **kw)
    rhs = 2.0 * oracle_mod.solve(f1, **kw) - 0.5 * oracle_mod.solve(f2, **kw)
    assert np.abs(lhs - rhs).max() < 1e-12 * np.abs(lhs).max()


def test_error_ratio_improves_with_buffers(oracle_mod):
    n = 128
    f, uex = inputs.manufactured(n, 0)
    e_conv = np.abs(oracle_mod.solve(f) - uex).max()
    er = {}
    for A, B in [(2, 0), (4, 1), (8, 0), (8, 2)]:
        u = oracle_mod.solve(f, seg=32, K=3, A=A, B=B)
        er[(A, B)] = np.abs(u - uex).max() / e_conv
    assert er[(2, 0)] > er[(4, 1)] > er[(8, 0)] > er[(8, 2)] >= 0.99
    assert er[(8, 2)] < 1.1  # acceptable in the sense of Sec. 5.2 (within ~10%)


def test_mbs_schedule(oracle_mod):
    """Sec. 5.2.1: the coarser compute region is the whole support of the
    finer one, so each level's buffer is twice the next coarser one's (in that
    level's cells); it is the largest schedule the geometry check accepts."""
    assert oracle_mod.mbs_schedule(4, 4) == [4, 8, 16, 32]
    assert oracle_mod.mbs_schedule(2, 1) == [2]
    J = oracle_mod.mbs_schedule(4, 3)
    assert oracle_mod.check_config(n=64, seg=16, K=3, J=J) == 0
    assert oracle_mod.check_config(n=64, seg=16, K=3, J=[J[0], J[1] + 2, J[2]]) != 0


def test_mbs_error_ratio_trends(oracle_mod):
    """Table 3's trend under the maximum buffer schedule: at fixed K and J_1
    the error ratio falls as the segments grow (larger N_0^V), and at fixed
    segments it falls as J_1 grows; MBS is never worse than the constant
    schedule with the same J_1 here."""
    n, K = 128, 2
    f, uex = inputs.manufactured(n, 0)
    e_conv = np.abs(oracle_mod.solve(f) - uex).max()

    def e_r(seg, J):
        return np.abs(oracle_mod.solve(f, seg=seg, K=K, J=J) - uex).max() / e_conv

    by_seg = [e_r(seg, oracle_mod.mbs_schedule(2, K)) for seg in (16, 32, 64)]
    assert by_seg[0] > by_seg[1] > by_seg[2] > 1.0
    mbs4 = e_r(32, oracle_mod.mbs_schedule(4, K))
    assert mbs4 < by_seg[1]
    assert mbs4 <= e_r(32, [4, 4]) * (1 + 1e-12)


def test_rejects_inconsistent_geometry(oracle_mod):
    assert oracle_mod.check_config(n=32, seg=12, K=2, J=[2, 2]) != 0   # seg does not divide n
    assert oracle_mod.check_config(n=32, seg=8, K=4, J=[2] * 4) != 0   # seg not divisible by 2^K
    assert oracle_mod.check_config(n=32, seg=8, K=2, J=[3, 4]) != 0    # odd buffer
    assert oracle_mod.check_config(n=32, seg=8, K=2, J=[2, 8]) != 0    # J_1 < J_2 / 2
    assert oracle_mod.check_config(n=32, seg=8, K=2, J=[4, 8]) == 0


@pytest.mark.parametrize("nc,J", [(8, [4, 4]), (16, [4, 4]), (16, [4, 6])])
def test_deep_coarse_solve_matches_masked_implementation(oracle_mod, nc, J):
    """SR with an exact coarsest solve at 8^3 (global V-cycle on 16^3) or at
    16^3 (the transition level itself) against the masked implementation."""
    n, seg, K = 64, 32, 2
    f, _ = inputs.manufactured(n, 2)
    a = oracle_mod.solve(f, seg=seg, K=K, J=J, n_coarse=nc)
    b = sr_masked.sr_fmg(f, seg, K, J, sr_masked.Params(), coarsest=nc)
    assert not np.isnan(b).any()
    assert np.abs(a - b).max() <= 1e-13 * np.abs(a).max()


def test_benchmark_configuration_at_discretisation_error(oracle_mod):
    """The benchmarked SR configuration on the oracle: 256^3, 512 segments of
    32^3, K = 3, J = (12, 12, 10), coarsest grid 16^3.  Plain FMG on that
    hierarchy is well below the discretisation error, the SR result stays
    within 0.05 e_disc of it (so e_r <= 1.1, the paper's acceptability
    threshold, Sec. 5.2, whatever the signs), while J = 8 adds about half an
    e_disc of its own."""
    n = 256
    kw = workloads.config(workloads.SR256)
    assert oracle_mod.buffer_schedule(kw["A"], kw["B"], kw["K"]) == [12, 12, 10]
    f, uex = inputs.manufactured(n, 0)
    uh = exact.dst_solve(f)
    e_disc = np.abs(uh - uex).max()
    plain = oracle_mod.solve(f, **workloads.config(workloads.PLAIN256))
    sr = oracle_mod.solve(f, **kw)
    assert np.abs(plain - uh).max() < 0.2 * e_disc
    assert np.abs(sr - uh).max() < 0.25 * e_disc
    assert np.abs(sr - plain).max() < 0.05 * e_disc
    assert np.abs(sr - uex).max() / np.abs(plain - uex).max() <= 1.1
    sr8 = oracle_mod.solve(f, seg=32, K=3, J=[8, 8, 8], n_coarse=16)
    assert np.abs(sr8 - plain).max() > 0.3 * e_disc
