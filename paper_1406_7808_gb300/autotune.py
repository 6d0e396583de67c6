"""Autotuner for the batched solves: per grid size the segment shape, the
coarsest exact grid and the kernels' launch shape; for the whole batch the
branch count of the CUDA graph.

- Segment shapes change the numerical result (segmental refinement trades
  buffer work for accuracy), so a candidate is eligible only if its measured
  error ratio e_r = |u_SR - u| / |u_plain - u| on the manufactured problem of
  that size stays at most `max_er` (the paper's acceptability threshold is
  about 1.1, Sec. 5.2), both solves at discretisation error: the coarsest
  grid is the deepest one the size halves to within 16^3 (16^3 for 64^3,
  128^3 and 256^3, 12^3 for 192^3), solved exactly.  Among eligible
  candidates the fastest solve wins.
- Launch shapes (cells in z per thread of the column kernels, cells per
  thread of the per-cell kernels) do not change a bit of the result; the
  fastest by timing wins.
- The graph's branch count does not change results; sr_fmg_batch_autotune
  picks it by timing.

Every timing and every solve runs through the C ABI.
"""
import numpy as np

from . import inputs, srfmg, workloads

# launch shapes tried per grid size: (zchunk, cells per thread)
SHAPES = [(8, 1), (8, 2), (16, 1), (16, 2), (16, 4), (32, 2), (32, 4)]


def deepest_coarse(n, limit=16):
    """Largest c <= limit with n = c 2^m, c >= 2 (the exact coarsest grid)."""
    c = n
    while c > limit:
        if c % 2:
            return 0
        c //= 2
    return c if c >= 2 else 0


def _time_solver(solver, ft, ut, reps):
    import torch
    for _ in range(2):
        solver.solve_async(ft, ut)
    solver.check()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        solver.solve_async(ft, ut)
    e1.record()
    torch.cuda.synchronize()
    solver.check()
    return e0.elapsed_time(e1) / reps


def tune_segments(n, candidates=None, common=None, max_er=1.1, reps=3):
    """Return (best keyword arguments, table of (kw, ms, e_r)) for grid n."""
    import torch
    if common is None:
        common = dict(A=8, B=0, mixed=True, n_outer=2, n_coarse=deepest_coarse(n))
    common = dict(common)
    candidates = candidates or workloads.SEGMENT_CANDIDATES.get(n, [dict()])
    f, uex = inputs.manufactured(n, 0)
    ft = torch.from_numpy(f).cuda()
    ut = torch.empty_like(ft)
    plain_kw = {k: v for k, v in common.items() if k not in ("A", "B")}
    with srfmg.Solver(n, **plain_kw) as s:
        s.solve(ft, ut)
        e_plain = float(np.abs(ut.cpu().numpy() - uex).max())
    table = []
    for cand in candidates:
        kw = dict(common, **cand)
        try:
            with srfmg.Solver(n, **kw) as s:
                ms = _time_solver(s, ft, ut, reps)
                e_r = float(np.abs(ut.cpu().numpy() - uex).max()) / e_plain
        except srfmg.SRFMGError:
            continue
        table.append((cand, ms, e_r))
    ok = [t for t in table if t[2] <= max_er]
    pick = min(ok, key=lambda t: t[1]) if ok else min(table, key=lambda t: t[2])
    return dict(common, **pick[0]), table


def tune_shape(n, kw, shapes=SHAPES, reps=3):
    """Fastest launch shape for a solver of grid n with keyword arguments kw;
    returns ((zchunk, cells per thread), {shape: ms})."""
    import torch
    f, _ = inputs.manufactured(n, 0)
    ft = torch.from_numpy(f).cuda()
    ut = torch.empty_like(ft)
    times = {}
    with srfmg.Solver(n, **kw) as s:
        for shape in shapes:
            s.set_launch_shape(*shape)
            times[shape] = _time_solver(s, ft, ut, reps)
    return min(times, key=times.get), times


def tuned_batch(problems, common=None, max_er=1.1, shapes=SHAPES):
    """Solvers for [(n, seed)] with tuned segment and launch shapes per size;
    returns (solvers, choices {n: (kw, segment table, launch shape, shape
    times)})."""
    choices = {}
    for n in sorted({n for n, _ in problems}):
        kw, table = tune_segments(n, common=common, max_er=max_er)
        shape, times = tune_shape(n, kw, shapes) if shapes else ((16, 2), {})
        choices[n] = (kw, table, shape, times)
    solvers = []
    for n, _ in problems:
        s = srfmg.Solver(n, **choices[n][0])
        s.set_launch_shape(*choices[n][2])
        solvers.append(s)
    return solvers, choices
