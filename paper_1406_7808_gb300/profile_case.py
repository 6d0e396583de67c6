"""Small, self-contained launches of the solver's kernels for profiler
captures (ncu): each case runs a fixed, seeded workload once and exits.

  python -m paper_1406_7808_gb300.profile_case smooth --n 256
      one Chebyshev degree-2 smoothing of a whole n^3 grid (two kernels:
      cheb_residual, cheb2_update)
  python -m paper_1406_7808_gb300.profile_case solve --n 256 [--plain] [--mixed] [--warmup 1]
          [--seg 32 --K 3 --A 11 --B 1 --n-coarse 16]
      warm-up solves then one solve of an SR configuration (default: the
      benchmark's segments, buffers and coarsest grid; --plain without
      segments; --mixed in the mixed-precision mode; --legs with the
      segment-resident legs)
  python -m paper_1406_7808_gb300.profile_case smooth27 --n 256
      one degree-2 smoothing with the 27-point operator ((14,3,1)/30) on the
      paper's domain [0,2]x[0,1]^2 with n cells per unit length (two
      column-form kernels)
"""
import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main():
    import torch

    from paper_1406_7808_gb300 import build, inputs, srfmg, workloads

    sr = workloads.SR256
    p = argparse.ArgumentParser()
    p.add_argument("case", choices=["smooth", "solve", "smooth27"])
    p.add_argument("--n", type=int, default=256)
    p.add_argument("--plain", action="store_true")
    p.add_argument("--mixed", action="store_true")
    p.add_argument("--warmup", type=int, default=1)
    p.add_argument("--seg", type=int, default=sr["seg"])
    p.add_argument("--K", type=int, default=sr["K"])
    p.add_argument("--A", type=int, default=sr["A"])
    p.add_argument("--B", type=int, default=sr["B"])
    p.add_argument("--n-coarse", type=int, default=sr["n_coarse"])
    p.add_argument("--legs", action="store_true",
                   help="segment-resident legs on (mixed mode; off by default)")
    a = p.parse_args()
    build.build()
    torch.cuda.set_device(0)
    if a.case == "smooth27":
        f, _ = inputs.paper_problem(a.n)
        ft = torch.from_numpy(f).cuda()
        u = torch.zeros_like(ft)
        srfmg.op_smooth(u, ft, 2, lengths=(2, 1, 1), stencil=27)
        torch.cuda.synchronize()
        return
    f, _ = inputs.manufactured(a.n, 0)
    ft = torch.from_numpy(f).cuda()
    if a.case == "smooth":
        u = torch.zeros_like(ft)
        srfmg.op_smooth(u, ft, 2)
    else:
        kw = dict(n_coarse=a.n_coarse)
        if not a.plain:
            kw.update(seg=a.seg, K=a.K, A=a.A, B=a.B)
        if a.mixed:
            kw["mixed"] = True
        with srfmg.Solver(a.n, **kw) as s:
            if a.legs:
                s.debug_segment_legs(True)
            ut = torch.empty_like(ft)
            for _ in range(a.warmup):
                s.solve_async(ft, ut)
            s.check()
            s.solve(ft, ut)
            print(f"launches per solve: {s.launches_per_solve}")
    torch.cuda.synchronize()


if __name__ == "__main__":
    main()
