#!/usr/bin/env python
"""Benchmark: segmental-refinement FMG (FP64) on a 256^3 Poisson problem at
discretisation error.

One step = one full SR-FMG solve (every step of the method: f hierarchy,
global FMG from the exactly solved 16^3 grid to the 32^3 transition level,
K = 3 SR stages over 512 segments of 32^3 genuine cells with J = (12, 12, 10)
buffer cells per side, output) of A u = f with the seeded manufactured
right-hand side.  Metric: fine-grid DOF/s = n^3 / time per solve (whole job:
all ranks' DOF over the slowest rank's time).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Rank 0 prints one JSON line.  --impl reference times the CPU oracle (the
plain C implementation the tests compare with) on this host's cores instead.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1406_7808_gb300 import workloads  # noqa: E402  (configuration only)

METRIC = "3D Poisson FMG fine-grid DOF/s, SR vs plain, at discretization error; %HBM peak"
N = workloads.SR256["n"]
SR = workloads.config(workloads.SR256)
PLAIN = workloads.config(workloads.PLAIN256)
SR_DEPTH2 = workloads.config(workloads.SR256_DEPTH2)
SEED = 0
VSOLVE_RTOL = 1e-4  # relative residual of the V-cycle comparison solver (Sec. 5.3)
# float64 FMA lanes per clock per SM on GB300 (the derived peak, reported
# beside the measured one)
FP64_LANES_PER_CLK_SM = 2


def workload_name(n=N, sr=SR):
    J = [2 * ((sr["A"] + sr["B"] * (sr["K"] - k)) // 2) for k in range(1, sr["K"] + 1)]
    nseg = (n // sr["seg"]) ** 3
    nc = sr.get("n_coarse", 0) or 2
    return (f"SR-FMG FP64 {n}^3 cells, {nseg} segments of {sr['seg']}^3, K={sr['K']} SR levels, "
            f"buffers Eq.(eq:nb) A={sr['A']} B={sr['B']} (J={J}), F(1,2,2) Chebyshev, "
            f"global levels {n >> sr['K']}^3..{nc}^3, {nc}^3 solved exactly"), J


def bench_config(world):
    """The workload's config, the same on both arms of the benchmark."""
    name, J = workload_name()
    return {"workload": name, "n": N, **SR, "J": J,
            "parallelism": "replicas" if world > 1 else "single",
            "l2": "inputs larger than L2: f is 134 MB and each solve moves about 21.6 GB "
                  "through DRAM (ncu)"}


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the mixed-precision and batched measurements")
    p.add_argument("--shard", action="store_true",
                   help="split one problem's segments among the ranks (redundant coarse "
                        "solves, one all-reduce of the transition level per SR stage) "
                        "instead of one replica per rank")
    return p.parse_args()


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.1)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self, min_mhz_under_load=300):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                rows.append((float(parts[0]), float(parts[1]), parts[3:7]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i, v in enumerate(r)
                          if v.lower().startswith("active")})
        loaded = [r[0] for r in rows if r[0] >= min_mhz_under_load] or [r[0] for r in rows]
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------

def ncu_traffic(kernel):
    """DRAM traffic per launch of `kernel` from the committed ncu summary, if
    the kernel source is unchanged since the capture (else None)."""
    path = os.path.join(ROOT, "profiles", f"ncu_{kernel}.md")
    csrc = os.path.join(ROOT, "paper_1406_7808_gb300", "csrc")
    srcs = [os.path.join(csrc, "kernels.cu"), os.path.join(csrc, "srfmg_device.cuh")]
    if not os.path.exists(path) or not all(os.path.exists(x) for x in srcs):
        return None
    sha = hashlib.sha256(b"".join(open(x, "rb").read() for x in srcs)).hexdigest()[:16]
    vals = {}
    for line in open(path):
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernels.cu + srfmg_device.cuh sha256[:16]") != sha:
        return None
    try:
        return float(vals["dram bytes per launch (scaled to the bench workload)"])
    except (KeyError, ValueError):
        return None


def csrc_sha():
    """sha256[:16] over the library's .cu and .cuh sources that the measured
    7-point solves run, concatenated in file-name order (the 27-point
    operator's kernels, kernels27.cu, are left out)."""
    d = os.path.join(ROOT, "paper_1406_7808_gb300", "csrc")
    names = sorted(x for x in os.listdir(d)
                   if x.endswith((".cu", ".cuh")) and x != "kernels27.cu")
    return hashlib.sha256(b"".join(open(os.path.join(d, x), "rb").read()
                                   for x in names)).hexdigest()[:16]


def ncu_dram_per_solve():
    """{workload: DRAM bytes per solve} from the committed ncu launch lists of
    whole solves, if the library sources are unchanged since (else {})."""
    path = os.path.join(ROOT, "profiles", "ncu_dram_per_solve.md")
    if not os.path.exists(path):
        return {}
    vals = {}
    for line in open(path):
        if ": " in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(": ", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("csrc sha256[:16]") != csrc_sha():
        return {}
    out = {}
    for k, v in vals.items():
        if k.endswith(" dram bytes per solve"):
            try:
                out[k[: -len(" dram bytes per solve")]] = float(v)
            except ValueError:
                pass
    return out


def dram_rate(nbytes, ms, hbm_peak):
    """Measured DRAM traffic of a solve against the measured copy bandwidth
    and the 8 TB/s nominal figure."""
    if not nbytes:
        return None
    gbs = nbytes / (ms / 1e3) / 1e9
    return {"dram_bytes_per_solve": nbytes, "gbs": gbs,
            "frac_of_measured": gbs / hbm_peak if hbm_peak else None,
            "frac_of_nominal_8tbs": gbs / 8000.0,
            "source": "profiles/ncu_dram_per_solve.md (ncu, whole solve)"}


def cpu_baseline(f, min_seconds=10.0, max_solves=6):
    """The oracle, as it stands, timed on this host's cores (full solves of
    the same workload until about min_seconds of work)."""
    import oracle
    threads = os.cpu_count() or 1
    times, u = [], None
    t_start = time.perf_counter()
    while len(times) < max_solves:
        t0 = time.perf_counter()
        u = oracle.solve(f, n_threads=threads, **SR)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start >= min_seconds:
            break
    mean = sum(times) / len(times)
    # one more solve on a single thread (the oracle's segment loop serialised)
    t0 = time.perf_counter()
    oracle.solve(f, n_threads=1, **SR)
    single = time.perf_counter() - t0
    return u, {"value": N ** 3 / mean, "unit": "DOF/s", "cores": threads, "kind": "oracle",
               "single_thread_dof_s": N ** 3 / single,
               "sample": f"{len(times)} full {N}^3 SR-FMG oracle solves (same f and geometry), "
                         f"OpenMP over segments, mean {mean:.2f} s per solve; plus one "
                         f"single-thread solve ({single:.2f} s)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_1406_7808_gb300 import inputs
    from oracle import build as oracle_build
    oracle_build.build()
    threads = os.cpu_count() or 1
    f, _ = inputs.manufactured(N, SEED)
    # a step is one full solve unless the whole run would take too long, then
    # the same segment geometry on a 128^3 grid (1/8 of the work)
    t0 = time.perf_counter()
    oracle.solve(f, n_threads=threads, **SR)
    t_full = time.perf_counter() - t0
    n_step, fs = N, f
    if (args.steps + args.warmup) * t_full > 180.0:
        n_step = N // 2
        fs, _ = inputs.manufactured(n_step, SEED)
    for _ in range(max(args.warmup - 1, 0)):
        oracle.solve(fs, n_threads=threads, **SR)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve(fs, n_threads=threads, **SR)
    dt = (time.perf_counter() - t0) / args.steps
    value = n_step ** 3 / dt
    sample = (f"one full {n_step}^3 SR-FMG oracle solve per step "
              f"({'the workload itself' if n_step == N else 'same segment geometry at 1/8 size'})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": threads, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def max_over_ranks(x, world, device="cuda"):
    """Largest value of x over the ranks of the job (the slowest rank's time);
    x itself on a single rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, seconds):
    """Whole-job throughput: every rank processes units_per_rank (replicas,
    weak scaling), the job takes the slowest rank's time."""
    return world * units_per_rank / seconds


def rank_seed(rank):
    """Seed of the manufactured problem a rank solves (replica r: seed r)."""
    return SEED + rank


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1406_7808_gb300 import build, inputs, srfmg, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def ranks_max(x):
        return max_over_ranks(x, world)

    # replicas: every rank solves its own instance (seeded by rank); no data
    # is exchanged between ranks
    f, u_exact = inputs.manufactured(N, rank_seed(rank))
    ft = torch.from_numpy(f).cuda()
    ut = torch.empty_like(ft)
    stream = torch.cuda.current_stream()

    def timed(solver, steps, sampler=None):
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ctx = sampler if sampler is not None else _Null()
        with ctx:
            e0.record(stream)
            for _ in range(steps):
                solver.solve_async(ft, ut)
            e1.record(stream)
            torch.cuda.synchronize()
        solver.check()
        barrier()
        return ranks_max(e0.elapsed_time(e1))

    # graph mode: each solve is one captured CUDA graph (same kernels)
    sr = srfmg.Solver(N, graph=True, **SR)
    for _ in range(args.warmup):
        sr.solve_async(ft, ut)
    sr.check()
    u_sr = ut.cpu().numpy()
    # measured FMA peaks of this device (the float64 one is the roofline's
    # denominator for the float64-pipe-bound kernels)
    fp64_peak = srfmg.probe_fma_rate(64) / 1e12
    fp32_peak = srfmg.probe_fma_rate(32) / 1e12
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    sampler = ClockSampler(local)
    total_ms = timed(sr, args.steps, sampler)
    clocks = sampler.summary()
    ms = total_ms / args.steps
    value = job_rate(N ** 3, world, ms / 1e3)
    launches = sr.launches_per_solve

    # per-kernel device times (a profiled repeat of the timed loop)
    sr.profile(True)
    for _ in range(args.steps):
        sr.solve_async(ft, ut)
    sr.check()
    prof = sr.profile_read()
    sr.profile(False)
    dominant = max(prof, key=lambda k: prof[k]["ms"])
    d = prof[dominant]
    achieved = d["ops"] / (d["ms"] / 1e3) / 1e12
    hbm_peak = None
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
    except (OSError, ValueError, KeyError):
        pass
    max_mhz = (clocks or {}).get("sm_max_mhz") or 2070.0
    fp64_derived = FP64_LANES_PER_CLK_SM * sms * max_mhz * 1e6 / 1e12
    roofline = {"bound": "alu", "kernel": dominant, "achieved": achieved,
                "peak": fp64_peak, "unit": "TFP64op/s", "frac": achieved / fp64_peak,
                "traffic": ncu_traffic(dominant),
                "peak_note": (f"measured: sr_probe_fma_rate(64) on this GPU, {fp64_peak:.3f} T "
                              f"FP64 FMA lane-op/s; derived 2 lanes/clk/SM x {sms} SMs x "
                              f"{max_mhz:.0f} MHz = {fp64_derived:.3f}"),
                "frac_of_derived": achieved / fp64_derived,
                "launches": d["launches"] // args.steps,
                "fp64_ops_per_launch": d["ops"] / d["launches"],
                "ms_per_launch": d["ms"] / d["launches"],
                "hbm_gbs": d["bytes"] / (d["ms"] / 1e3) / 1e9,
                "hbm_frac_of_measured": (d["bytes"] / (d["ms"] / 1e3) / 1e9 / hbm_peak)
                if hbm_peak else None}
    kernels = {k: {"ms_per_solve": v["ms"] / args.steps,
                   "share": v["ms"] / sum(x["ms"] for x in prof.values()),
                   "tfp64ops": v["ops"] / (v["ms"] / 1e3) / 1e12 if v["ms"] else None}
               for k, v in sorted(prof.items(), key=lambda kv: -kv[1]["ms"])}

    # the same solve launched kernel by kernel (no graph)
    direct = srfmg.Solver(N, **SR)
    for _ in range(args.warmup):
        direct.solve_async(ft, ut)
    direct.check()
    direct_ms = timed(direct, args.steps) / args.steps
    direct.close()

    # the same solve without segmental refinement (plain FMG), same f
    plain = srfmg.Solver(N, graph=True, **PLAIN)
    for _ in range(args.warmup):
        plain.solve_async(ft, ut)
    plain.check()
    u_plain = ut.cpu().numpy()
    plain_ms = timed(plain, args.steps) / args.steps
    plain_bytes = profiled_bytes(plain, ft, ut)
    # the paper's comparison solver: V-cycles from zero to a relative
    # residual of 1e-4 (Sec. 5.3), same f
    vs = None
    if not args.no_extras:
        plain.vsolve(ft, ut.zero_(), rtol=VSOLVE_RTOL)
        barrier()
        vstate = {}

        def vstep():
            _, vstate["cycles"], vstate["rel"] = plain.vsolve(ft, ut.zero_(), rtol=VSOLVE_RTOL)
        vs_ms = ranks_max(_time_loop(vstep, args.steps, stream)) / args.steps
        vs = {"rtol": VSOLVE_RTOL, "ms": vs_ms, "dof_s": world * N ** 3 / (vs_ms / 1e3),
              "cycles": vstate["cycles"], "rel_resid": vstate["rel"],
              "e": float(np.abs(ut.cpu().numpy() - u_exact).max())}
    plain.close()
    sr_bytes = sum(v["bytes"] for v in prof.values()) / args.steps

    # end to end through the C ABI from pinned host memory: every step copies
    # its f in and its u out; consecutive steps overlap their copies with
    # each other's solves (sr_fmg_solve_host_async)
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    for _ in range(2):
        sr.solve_host_async(fh, uh)
    sr.check_host()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        sr.solve_host_async(fh, uh)
    sr.check_host()
    e2e_s = ranks_max(time.perf_counter() - t0) / args.steps
    sr.close()
    del fh, uh

    # the same segments at the paper's depth (2^3 coarsest grid, J = 8) and
    # plain FMG there: far from discretisation error (comparison only)
    depth2 = {}
    for kind, kw in (("sr", SR_DEPTH2), ("plain", {})):
        with srfmg.Solver(N, graph=True, **kw) as s2:
            for _ in range(args.warmup):
                s2.solve_async(ft, ut)
            s2.check()
            depth2[kind + "_u"] = ut.cpu().numpy()
            depth2[kind + "_ms"] = timed(s2, args.steps) / args.steps

    mixed = batch = None
    paper = adjoint = None
    if not args.no_extras:
        mixed = measure_mixed(args, timed_fn=ranks_max, world=world, rank=rank)
        batch = measure_batch(args, ranks_max, world)
        paper = measure_paper(args, ranks_max, world, fp64_peak)
        adjoint = measure_adjoint(args, ranks_max, world, rank)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    # accuracy at discretisation level
    acc = {}
    try:
        from scipy.fft import dstn, idstn
        k = np.arange(1, N + 1)
        l1 = 4.0 * N * N * np.sin(k * np.pi / (2.0 * N)) ** 2
        lam = l1[:, None, None] + l1[None, :, None] + l1[None, None, :]
        u_h = idstn(dstn(f, type=2, workers=os.cpu_count()) / lam, type=2,
                    workers=os.cpu_count())
        acc["e_disc"] = float(np.abs(u_h - u_exact).max())
        acc["e_alg_sr"] = float(np.abs(u_sr - u_h).max())
        acc["e_alg_plain"] = float(np.abs(u_plain - u_h).max())
        acc["e_alg_sr_over_e_disc"] = acc["e_alg_sr"] / acc["e_disc"]
        acc["e_alg_plain_over_e_disc"] = acc["e_alg_plain"] / acc["e_disc"]
        acc["sr_minus_plain_over_e_disc"] = float(np.abs(u_sr - u_plain).max()) / acc["e_disc"]
        for kind in ("sr", "plain"):
            depth2["e_alg_" + kind + "_over_e_disc"] = \
                float(np.abs(depth2[kind + "_u"] - u_h).max()) / acc["e_disc"]
    except ImportError:
        pass
    acc["e_sr"] = float(np.abs(u_sr - u_exact).max())
    acc["e_plain"] = float(np.abs(u_plain - u_exact).max())
    acc["e_r"] = acc["e_sr"] / acc["e_plain"]
    e_d2 = {k: float(np.abs(depth2.pop(k + "_u") - u_exact).max()) for k in ("sr", "plain")}
    depth2.update({"e_r": e_d2["sr"] / e_d2["plain"], "config": dict(SR_DEPTH2),
                   "sr_dof_s": world * N ** 3 / (depth2["sr_ms"] / 1e3),
                   "plain_dof_s": world * N ** 3 / (depth2["plain_ms"] / 1e3)})
    if vs is not None:
        vs["e_over_e_plain_fmg"] = vs["e"] / acc["e_plain"]

    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        u_or, cpu = cpu_baseline(f)
        acc["max_rel_diff_vs_oracle"] = float(np.abs(u_sr - u_or).max() / np.abs(u_or).max())

    if mixed is not None and world == 1 and not args.no_cpu_baseline:
        import oracle
        mf, _ = inputs.manufactured(mixed["n"], 1)
        okw = {k: v for k, v in workloads.config(workloads.MIXED512).items()
               if k not in ("mixed", "n_outer")}
        ref = oracle.solve_refined(mf, workloads.MIXED512["n_outer"], n_threads=os.cpu_count(),
                                   **okw)
        diff = float(np.abs(mixed.pop("u") - ref).max())
        h = 1.0 / mixed["n"]
        e_disc = abs(np.pi ** 2 * h * h / (4 * np.sin(np.pi * h / 2) ** 2) - 1) * \
            np.cos(np.pi * h / 2) ** 3
        mixed["max_abs_diff_vs_oracle_fp64_loop"] = diff
        mixed["bound"] = "0.1 e_disc"
        mixed["e_disc"] = float(e_disc)
        mixed["within_bound"] = bool(diff <= 0.1 * e_disc)
    elif mixed is not None:
        mixed.pop("u", None)
    hbm = hbm_peak or None
    comparison = {
        "plain_fmg_fp64_256": {"dof_s": world * N ** 3 / (plain_ms / 1e3), "ms": plain_ms,
                               "hbm_gbs": plain_bytes / (plain_ms / 1e3) / 1e9,
                               "hbm_frac_of_measured": plain_bytes / (plain_ms / 1e3) / 1e9 / hbm
                               if hbm else None},
        "sr_fmg_fp64_256_kernel_by_kernel": {"ms": direct_ms,
                                             "dof_s": world * N ** 3 / (direct_ms / 1e3)},
        "paper_problem_27pt": paper,
        "sr_fmg_fp64_256": {"dof_s": value, "ms": ms,
                            "hbm_gbs": sr_bytes / (ms / 1e3) / 1e9,
                            "hbm_frac_of_measured": sr_bytes / (ms / 1e3) / 1e9 / hbm
                            if hbm else None},
        "vcycle_solve_fp64_256": vs,
        "paper_depth_2cubed_fp64_256": depth2,
        "mixed_sr_512": mixed,
        "batched_mixed": batch,
        "adjoint_sr_fp64_256": adjoint,
    }
    if mixed is not None and hbm:
        mixed["hbm_frac_of_measured"] = mixed["hbm_gbs"] / hbm
    dram = ncu_dram_per_solve()
    comparison["plain_fmg_fp64_256"]["dram"] = dram_rate(dram.get("plain_fmg_fp64_256"),
                                                         plain_ms, hbm_peak)
    comparison["sr_fmg_fp64_256"]["dram"] = dram_rate(dram.get("sr_fmg_fp64_256"), ms, hbm_peak)
    if mixed is not None:
        mixed["dram"] = dram_rate(dram.get("mixed_sr_512"), mixed["ms"], hbm_peak)

    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": bench_config(world),
        "e2e": {"value": world * N ** 3 / e2e_s, "unit": "DOF/s",
                "h2d_bytes_per_step": N ** 3 * 8, "d2h_bytes_per_step": N ** 3 * 8},
        "gpu_launches": launches * args.steps,
        "roofline": roofline,
        "hbm": comparison["sr_fmg_fp64_256"]["dram"],
        "peaks": {"fp64_fma_tops_measured": fp64_peak, "fp32_fma_tops_measured": fp32_peak,
                  "fp64_fma_tops_derived": fp64_derived, "sms": sms,
                  "hbm_gbs_measured": hbm_peak},
        "cpu_baseline": cpu,
        "clocks": clocks,
        "accuracy": acc,
        "kernels": kernels,
        "comparison": comparison,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_sharded(args):
    """One 256^3 problem, its 512 segments split into contiguous ranges, one
    per rank; every rank holds the whole f and solves the transition level and
    below redundantly; per SR stage one all-reduce (sum) of the two
    transition-level arrays (32^3 doubles each) over NCCL.  value = n^3 /
    the slowest rank's time per solve (strong scaling of one problem)."""
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1406_7808_gb300 import build, inputs, srfmg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        raise SystemExit("--warmup must be at least 3")
    build.build()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def allreduce(ts):
        for t in ts:
            dist.all_reduce(t)

    reduce_sum = allreduce if world > 1 else None
    nsegs = srfmg.segment_count(N, SR["seg"])
    first, count = srfmg.segment_range(nsegs, rank, world)
    f, u_exact = inputs.manufactured(N, SEED)
    ft = torch.from_numpy(f).cuda()
    ut = torch.zeros_like(ft)
    stream = torch.cuda.current_stream()
    solver = srfmg.Solver(N, segments=(first, count), **SR)

    def step():
        srfmg.solve_staged([solver], ft, ut, reduce_sum)

    for _ in range(args.warmup):
        step()
    solver.check()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    barrier()
    sampler = ClockSampler(local)
    with sampler:
        ms = _time_loop(step, args.steps, stream) / args.steps
    solver.check()
    launches = solver.launches_per_solve * args.steps
    ms = max_over_ranks(ms, world)
    clocks = sampler.summary()
    # end to end: f in from pinned host memory and this rank's u out, every step
    fh = torch.from_numpy(f).pin_memory()
    uh = torch.empty_like(fh).pin_memory()
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ft.copy_(fh, non_blocking=True)
        step()
        uh.copy_(ut, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, world) / args.steps
    # the whole solution (each cell written by one rank, the others zero)
    # and its error ratio against plain FMG on the same f
    if world > 1:
        dist.all_reduce(ut)
    u = ut.cpu().numpy()
    with srfmg.Solver(N, **PLAIN) as p:
        up = p.solve(ft).cpu().numpy()
    e_r = float(np.abs(u - u_exact).max() / np.abs(up - u_exact).max())
    solver.close()
    if rank == 0:
        name, J = workload_name()
        line = {"metric": METRIC, "value": N ** 3 / (ms / 1e3), "unit": "DOF/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": name, "n": N, **SR, "J": J,
                           "parallelism": f"segments split over {world} ranks, transition "
                                          f"level all-reduced per stage",
                           "l2": "inputs larger than L2: f is 134 MB"},
                "e2e": {"value": N ** 3 / e2e_s, "unit": "DOF/s",
                        "h2d_bytes_per_step": N ** 3 * 8, "d2h_bytes_per_step": N ** 3 * 8},
                "gpu_launches": launches, "clocks": clocks,
                "accuracy": {"e_r": e_r},
                "exchange_bytes_per_stage": 2 * (N >> SR["K"]) ** 3 * 8}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def profiled_bytes(solver, ft, ut, reps=2):
    """Algorithmic bytes of one solve, from the library's per-kernel profile."""
    solver.profile(True)
    for _ in range(reps):
        solver.solve_async(ft, ut)
    solver.check()
    prof = solver.profile_read()
    solver.profile(False)
    return sum(v["bytes"] for v in prof.values()) / reps


def _time_loop(step, steps, stream=None):
    import torch
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def measure_paper(args, timed_fn, world, fp64_peak):
    """The paper's own model problem (Sec. 5.1) at Table 2's N = 256 column:
    [0,2]x[0,1]^2 with 1024 x 512 x 512 cells, 27-point operator ((14,3,1)/30),
    4 x 2 x 2 segments of 256^3, K = 5, A = 8, B = 0; plain FMG on the same f.
    Reports both solves' times, the error ratio e_r against the exact u
    (the paper prints 1.13 for its stencil), and the FP64 rate of the
    dominant 27-point kernel from the library's per-kernel profile."""
    import numpy as np
    import torch
    from paper_1406_7808_gb300 import inputs, srfmg
    n = 512
    geo = dict(lengths=(2, 1, 1), stencil=27)
    f, u = inputs.paper_problem(n)
    ft = torch.from_numpy(f).cuda()
    ut = torch.empty_like(ft)
    out = {"grid": [1024, 512, 512], "segments": [4, 2, 2], "seg": 256, "K": 5, "A": 8, "B": 0,
           "weights": list(srfmg.W27_DEFAULT), "paper_e_r": 1.13}
    steps = max(2, min(args.steps, 5))
    err = {}
    for name, kw in (("sr", dict(seg=256, K=5, A=8, B=0)), ("plain", {})):
        with srfmg.Solver(n, graph=True, **geo, **kw) as s:
            for _ in range(3):
                s.solve_async(ft, ut)
            s.check()
            ms = timed_fn(_time_loop(lambda: s.solve_async(ft, ut), steps)) / steps
            s.check()
            err[name] = float(np.abs(ut.cpu().numpy() - u).max())
            out[name + "_ms"] = ms
            out[name + "_dof_s"] = world * f.size / (ms / 1e3)
            if name == "sr":
                s.profile(True)
                s.solve_async(ft, ut)
                s.check()
                prof = s.profile_read()
                s.profile(False)
                top = max(prof, key=lambda k: prof[k]["ms"])
                d = prof[top]
                out["dominant_kernel"] = {
                    "kind": top, "share": d["ms"] / sum(v["ms"] for v in prof.values()),
                    "tfp64ops": d["ops"] / (d["ms"] / 1e3) / 1e12,
                    "frac_of_fp64_peak": d["ops"] / (d["ms"] / 1e3) / 1e12 / fp64_peak}
    out["e_sr"], out["e_conv"] = err["sr"], err["plain"]
    out["e_r"] = err["sr"] / err["plain"]
    return out


def measure_mixed(args, timed_fn, world, rank):
    """Mixed-precision SR-FMG, 512^3 cells, 64^3-cell segments, K = 4 (f of
    the manufactured problem at seed 1)."""
    import numpy as np
    import torch
    from paper_1406_7808_gb300 import inputs, srfmg, workloads
    kw = workloads.MIXED512
    n = kw["n"]
    f, _ = inputs.manufactured(n, 1 + rank)
    ft = torch.from_numpy(f).cuda()
    ut = torch.empty_like(ft)
    with srfmg.Solver(n, graph=True, **workloads.config(kw)) as s:
        for _ in range(args.warmup):
            s.solve_async(ft, ut)
        s.check()
        u = ut.cpu().numpy()
        total = timed_fn(_time_loop(lambda: s.solve_async(ft, ut), args.steps))
        s.check()
        ms = total / args.steps
        nbytes = profiled_bytes(s, ft, ut)
    return {"n": n, "config": workloads.config(kw), "dof_s": world * n ** 3 / (ms / 1e3),
            "ms": ms, "hbm_gbs": nbytes / (ms / 1e3) / 1e9, "u": u}


def measure_adjoint(args, timed_fn, world, rank):
    """The differentiable solve at 256^3 (SR-FMG FP64, the benchmark's
    segments): one step = forward solve, loss 0.5 ||u - u_target||^2 and
    the backward pass (a second SR-FMG solve on u - u_target), through
    torch.autograd."""
    import torch
    from paper_1406_7808_gb300 import inputs, srfmg
    n = N
    ft = torch.from_numpy(inputs.manufactured(n, rank)[0]).cuda().requires_grad_(True)
    target = torch.from_numpy(inputs.target(n)).cuda()
    with srfmg.Solver(n, **SR) as s:
        def step():
            if ft.grad is not None:
                ft.grad = None
            u = srfmg.solve_autograd(ft, s)
            loss = 0.5 * ((u - target) ** 2).sum()
            loss.backward()
        for _ in range(max(1, args.warmup)):
            step()
        steps = max(2, min(args.steps, 5))
        total = timed_fn(_time_loop(step, steps))
        ms = total / steps
    return {"n": n, "config": dict(SR), "steps": steps, "ms_per_step": ms,
            "dof_s": world * n ** 3 / (ms / 1e3),
            "note": "forward + backward solves, loss and gradient on the device"}


def measure_batch(args, timed_fn, world):
    """64 right-hand sides (16 each of 64^3, 128^3, 192^3, 256^3), mixed
    precision, one CUDA graph launch per batch, the deepest exact coarsest
    grid each size allows, autotuned segment shapes, launch shapes and graph
    branches."""
    import torch
    from paper_1406_7808_gb300 import autotune, inputs, srfmg, workloads
    problems = workloads.batch_problems()
    solvers, choices = autotune.tuned_batch(problems)
    fs = [torch.from_numpy(inputs.manufactured(n, seed)[0]).cuda() for n, seed in problems]
    us = [torch.empty_like(f) for f in fs]
    b = srfmg.Batch(solvers)
    branches, _ = b.autotune(fs, us)
    for _ in range(args.warmup):
        b.solve_async(fs, us)
    b.check()
    steps = max(3, args.steps // 4)
    total = timed_fn(_time_loop(lambda: b.solve_async(fs, us), steps))
    b.check()
    ms = total / steps
    dof = sum(n ** 3 for n, _ in problems)
    b.close()
    for s in solvers:
        s.close()
    return {"problems": len(problems), "sizes": list(workloads.BATCH_SIZES),
            "dof_per_batch": dof, "ms_per_batch": ms, "dof_s": world * dof / (ms / 1e3),
            "graph_branches": branches, "timed_batches": steps,
            "choice": {str(n): {"seg": c[0].get("seg"), "K": c[0].get("K"),
                                "n_coarse": c[0].get("n_coarse"), "zchunk": c[2][0],
                                "cells_per_thread": c[2][1],
                                "segment_table": [[t[0], round(t[1], 3), round(t[2], 3)]
                                                  for t in c[1]],
                                "shape_ms": {f"{z},{p}": round(v, 3)
                                             for (z, p), v in c[3].items()}}
                       for n, c in choices.items()}}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *exc):
        return False


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.shard:
        run_sharded(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
