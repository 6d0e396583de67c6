"""Autotuner for the segment shape of each grid size and the branch count of
the batched CUDA graph.

Segment shapes change the numerical result (segmental refinement trades
buffer work for accuracy), so a candidate is eligible only if its measured
error ratio e_r = |u_SR - u| / |u_plain - u| on the manufactured problem of
that size stays at most `max_er` (the paper's acceptability threshold is
about 1.1, Sec. 5.2); among eligible candidates the fastest solve wins.  The
graph's branch count does not change results; sr_fmg_batch_autotune picks it
by timing.  Every timing and every solve runs through the C ABI.
"""
import numpy as np

from . import inputs, srfmg, workloads


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
    common = dict(A=8, B=0, mixed=True, n_outer=2) if common is None else dict(common)
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


def tuned_batch(problems, common=None, max_er=1.1):
    """Solvers for [(n, seed)] with tuned segment shapes per size; returns
    (solvers, choices {n: (kw, table)})."""
    choices = {}
    for n in sorted({n for n, _ in problems}):
        choices[n] = tune_segments(n, common=common, max_er=max_er)
    solvers = [srfmg.Solver(n, **choices[n][0]) for n, _ in problems]
    return solvers, choices
