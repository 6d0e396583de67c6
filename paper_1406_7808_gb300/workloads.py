"""Named workloads (grid sizes, segment geometry, buffer schedule, precision)
used by the benchmark, the smoke check and the tests.  Configuration only:
no arithmetic of the method lives here."""

# SR-FMG FP64 at discretisation error: 256^3 cells, 512 segments of 32^3,
# K = 3, buffers J = (12, 12, 10) (Eq. eq:nb with A = 11, B = 1), coarsest
# grid 16^3 solved exactly.  Plain FMG on this hierarchy leaves an algebraic
# error of about 0.13 e_disc, and these buffers keep the SR result within
# 0.04 e_disc of it (e_r about 0.97).
SR256 = dict(n=256, seg=32, K=3, A=11, B=1, n_coarse=16)
# plain FMG FP64 on the same grid and hierarchy
PLAIN256 = dict(n=256, n_coarse=16)
# the same segments at the paper's depth (coarsest grid 2^3) with J = 8:
# there FMG leaves about 10 e_disc of algebraic error in the smoothest mode
SR256_DEPTH2 = dict(n=256, seg=32, K=3, A=8, B=0)
PLAIN256_DEPTH2 = dict(n=256)
# mixed-precision SR-FMG: 512^3 cells, 512 segments of 64^3, K = 4, J = 8,
# coarsest grid 16^3 solved exactly (float64 arithmetic)
MIXED512 = dict(n=512, seg=64, K=4, A=8, B=0, mixed=True, n_outer=2, n_coarse=16)

# batched: 16 right-hand sides each of 64^3, 128^3, 192^3, 256^3 cells,
# mixed precision, manufactured f with seeds 100 + i
BATCH_SIZES = (64, 128, 192, 256)
BATCH_PER_SIZE = 16

# segment shapes the autotuner may choose from, per grid size (J = 8 buffer
# cells per side, Eq. eq:nb with A = 8, B = 0); a candidate whose
# transition level would lie below the exact coarsest grid is skipped
SEGMENT_CANDIDATES = {
    64: [dict(seg=16, K=2), dict(seg=32, K=2), dict(seg=32, K=3), dict(seg=64, K=4)],
    128: [dict(seg=16, K=2), dict(seg=32, K=3), dict(seg=64, K=3), dict(seg=64, K=4)],
    192: [dict(seg=32, K=3), dict(seg=64, K=4)],
    256: [dict(seg=32, K=3), dict(seg=64, K=4)],
}


def batch_problems(sizes=BATCH_SIZES, per_size=BATCH_PER_SIZE):
    """[(n, seed)] for the batched workload, sizes interleaved."""
    out = []
    i = 0
    for _ in range(per_size):
        for n in sizes:
            out.append((n, 100 + i))
            i += 1
    return out


def config(kw):
    """Solver keyword arguments without the grid size."""
    return {k: v for k, v in kw.items() if k != "n"}
